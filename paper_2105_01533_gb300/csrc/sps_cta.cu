// Small-state runs: one CTA applies a sequence of passes to a state of at most
// kSmallCap entries held in shared memory, so a chain of small passes costs one
// launch instead of one or two per pass.
//
// Branching passes here use the insert-once gather rule of Sec. 3.1: the CTA
// builds a table of its input labels (indices claimed with a 32-bit CAS, no
// amplitude atomics), every active entry looks up its partner (label with the
// gate's flip mask applied); if both are present only the entry whose selector
// bit is 1 writes the pair, computing M * (a0, a1) with each product and sum
// rounded once, as the scatter form does. Outputs are pruned and compacted with
// a block scan. Fused passes run the op list per entry.
#include <cuda_runtime.h>

#include <cstdint>

#include "sps_device.cuh"
#include "sps_internal.h"

namespace sps {
namespace {

using namespace dev;

constexpr uint32_t EMPTY_IDX = 0xFFFFFFFFu;

struct SmemSoA {
  uint64_t* lo;
  uint64_t* hi;
  double* re;
  double* im;
};

__device__ __forceinline__ SmemSoA smem_soa(unsigned char* base) {
  SmemSoA s;
  s.lo = reinterpret_cast<uint64_t*>(base);
  s.hi = s.lo + kSmallCap;
  s.re = reinterpret_cast<double*>(s.hi + kSmallCap);
  s.im = s.re + kSmallCap;
  return s;
}

// exclusive block scan of per-thread counts; returns the offset, *total the sum
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t incl = v;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, incl, d);
    if (lane >= (unsigned)d) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? warp_sums[lane] : 0u;
    uint32_t wi = w;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, wi, d);
      if (lane >= (unsigned)d) wi += t;
    }
    if (lane < nw) warp_sums[lane] = wi - w;
    if (lane == 31) warp_sums[32] = wi;
  }
  __syncthreads();
  const uint32_t off = warp_sums[warp] + incl - v;
  *total = warp_sums[32];
  __syncthreads();
  return off;
}

template <int KW>
__device__ __forceinline__ uint32_t lookup(const uint32_t* tab, const SmemSoA& a, uint64_t lo,
                                           uint64_t hi) {
  uint32_t h = (uint32_t)hash_label<KW>(lo, hi) & (kSmallTableSlots - 1);
  for (uint32_t p = 0; p < kSmallTableSlots; ++p, h = (h + 1) & (kSmallTableSlots - 1)) {
    const uint32_t j = tab[h];
    if (j == EMPTY_IDX) return EMPTY_IDX;
    if (a.lo[j] == lo && (KW == 1 || a.hi[j] == hi)) return j;
  }
  return EMPTY_IDX;
}

template <int KW>
__global__ void __launch_bounds__(kSmallThreads) k_small_run(Ctl* ctl, Bufs bufs,
                                                             const unsigned char* arena,
                                                             uint32_t pass_off, uint32_t npasses,
                                                             uint64_t capacity,
                                                             unsigned long long* plog) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemSoA A = smem_soa(smem);
  SmemSoA B = smem_soa(smem + 32 * kSmallCap);
  uint32_t* tab = reinterpret_cast<uint32_t*>(smem + 64 * kSmallCap);
  uint32_t* warp_sums = tab + kSmallTableSlots;   // 33 words
  if (ctl->status != 0u) return;
  const uint64_t n0 = ctl->nnz;
  const unsigned cur = ctl->cur;
  if (n0 > kSmallCap) {  // the host's bound said this cannot happen
    if (threadIdx.x == 0) fail(ctl, SPS_ERR_CAPACITY, 0u, 0ull);
    return;
  }
  const uint64_t cap = capacity < kSmallCap ? capacity : kSmallCap;
  uint32_t n = (uint32_t)n0;
  const SoA in = pick(bufs, cur);
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    A.lo[i] = in.lo[i];
    A.hi[i] = KW == 2 ? in.hi[i] : 0ull;
    A.re[i] = in.re[i];
    A.im[i] = in.im[i];
  }
  __syncthreads();
  const RunPass* passes = reinterpret_cast<const RunPass*>(arena + pass_off);
  const double r = 0.70710678118654752440;
  for (uint32_t pi = 0; pi < npasses; ++pi) {
    const RunPass rp = passes[pi];
    if (rp.kind == PASS_FUSED) {
      const FOp* ops = reinterpret_cast<const FOp*>(arena + rp.ops_off);
      const PhasePair* ph = reinterpret_cast<const PhasePair*>(arena + rp.ph_off);
      for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        uint64_t k0 = A.lo[i], k1 = A.hi[i];
        uint32_t cnt = 0;
        bool any = false;
        double acc_re = 1.0, acc_im = 0.0;
        for (uint32_t j = 0; j < rp.nops; ++j) {
          const FOp o = ops[j];
          bool cond = (k0 & o.c[0]) == o.c[0];
          if (KW == 2) cond = cond && ((k1 & o.c[1]) == o.c[1]);
          const bool sel = o.sbit != NO_SEL && label_bit(k0, k1, o.sbit);
          cnt += cond ? (sel ? o.a1 : o.a0) : 0u;
          if (o.ph != NO_PH && cond) {
            const PhasePair pp = ph[o.ph];
            const double pr = sel ? pp.re1 : pp.re0, pim = sel ? pp.im1 : pp.im0;
            const double nr = acc_re * pr - acc_im * pim;
            const double ni = acc_re * pim + acc_im * pr;
            acc_re = nr;
            acc_im = ni;
            any = true;
          }
          const uint64_t m = cond ? ~0ull : 0ull;
          k0 ^= o.t[0] & m;
          if (KW == 2) k1 ^= o.t[1] & m;
        }
        A.lo[i] = k0;
        A.hi[i] = k1;
        cnt &= 7u;
        if (cnt != 0u || any) {
          double re = A.re[i], im = A.im[i];
          if (any) {
            const double nr = re * acc_re - im * acc_im;
            const double ni = re * acc_im + im * acc_re;
            re = nr;
            im = ni;
          }
          if (cnt & 1u) {
            const double nr = r * (re - im);
            const double ni = r * (re + im);
            re = nr;
            im = ni;
          }
          switch (cnt >> 1) {
            case 1: { const double t = re; re = -im; im = t; break; }
            case 2: re = -re; im = -im; break;
            case 3: { const double t = re; re = im; im = -t; break; }
            default: break;
          }
          A.re[i] = re;
          A.im[i] = im;
        }
      }
      __syncthreads();
      continue;
    }
    // branching pass, gather form
    const BranchOp op = *reinterpret_cast<const BranchOp*>(arena + rp.br_off);
    for (uint32_t sl = threadIdx.x; sl < kSmallTableSlots; sl += blockDim.x) tab[sl] = EMPTY_IDX;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      uint32_t h = (uint32_t)hash_label<KW>(A.lo[i], A.hi[i]) & (kSmallTableSlots - 1);
      for (uint32_t p = 0; p < kSmallTableSlots; ++p, h = (h + 1) & (kSmallTableSlots - 1))
        if (atomicCAS(&tab[h], EMPTY_IDX, i) == EMPTY_IDX) break;
    }
    __syncthreads();
    // rounds of one input per thread; each input writes 0, 1 or 2 entries
    uint32_t base = 0;
    bool over = false;
    for (uint32_t r0 = 0; r0 < n; r0 += blockDim.x) {
      const uint32_t i = r0 + threadIdx.x;
      uint64_t l0 = 0, h0 = 0, l1 = 0, h1 = 0;
      double v0r = 0, v0i = 0, v1r = 0, v1i = 0;
      bool w0 = false, w1 = false;
      if (i < n) {
        const uint64_t k0 = A.lo[i], k1 = A.hi[i];
        const double re = A.re[i], im = A.im[i];
        bool active = (k0 & op.c[0]) == op.c[0] && (k1 & op.c[1]) == op.c[1];
        const bool x = label_bit(k0, k1, op.sbit);
        if (op.givens) active = active && (x != label_bit(k0, k1, op.qbit));
        if (!active) {
          l0 = k0; h0 = k1; v0r = re; v0i = im;
          w0 = keep_amp(re, im, rp.eps2, eps_pattern(rp.eps));
        } else {
          const uint64_t p0 = k0 ^ op.m[0], p1 = k1 ^ op.m[1];
          const uint32_t j = lookup<KW>(tab, A, p0, p1);
          if (j == EMPTY_IDX || x) {   // else the partner with selector bit 1 writes the pair
            const double pre = j != EMPTY_IDX ? A.re[j] : 0.0;
            const double pim = j != EMPTY_IDX ? A.im[j] : 0.0;
            // (a0, a1) on (label with selector 0, label with selector 1)
            const double a0r = x ? pre : re, a0i = x ? pim : im;
            const double a1r = x ? re : pre, a1i = x ? im : pim;
            l0 = x ? p0 : k0; h0 = x ? p1 : k1;
            l1 = x ? k0 : p0; h1 = x ? k1 : p1;
            pair_action(op, j != EMPTY_IDX, x, a0r, a0i, a1r, a1i, &v0r, &v0i, &v1r, &v1i);
            w0 = keep_amp(v0r, v0i, rp.eps2, eps_pattern(rp.eps));
            w1 = keep_amp(v1r, v1i, rp.eps2, eps_pattern(rp.eps));
          }
        }
      }
      uint32_t total = 0;
      const uint32_t off = base + block_scan((w0 ? 1u : 0u) + (w1 ? 1u : 0u), warp_sums, &total);
      if (base + total > cap) {
        over = true;
        break;
      }
      if (w0) {
        B.lo[off] = l0; B.hi[off] = h0; B.re[off] = v0r; B.im[off] = v0i;
      }
      if (w1) {
        const uint32_t o1 = off + (w0 ? 1u : 0u);
        B.lo[o1] = l1; B.hi[o1] = h1; B.re[o1] = v1r; B.im[o1] = v1i;
      }
      base += total;
    }
    if (over) {
      if (threadIdx.x == 0) fail(ctl, SPS_ERR_CAPACITY, rp.pass_serial, rp.fail_tag);
      __syncthreads();
      break;   // A still holds the state before this pass
    }
    __syncthreads();
    const uint32_t total = base;
    const SmemSoA t = A;
    A = B;
    B = t;
    n = total;
  }
  // publish: the state goes to the other global buffer
  const SoA out = pick(bufs, cur ^ 1u);
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    out.lo[i] = A.lo[i];
    if (KW == 2) out.hi[i] = A.hi[i];
    out.re[i] = A.re[i];
    out.im[i] = A.im[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    ctl->nnz = n;
    ctl->cur = cur ^ 1u;
    if (plog) {
      plog[0] = n0;
      plog[1] = n;
    }
  }
}

}  // namespace

int launch_small_run(void* stream, int key_words, Ctl* ctl, Bufs bufs, const unsigned char* arena,
                     uint32_t pass_off, uint32_t npasses, uint64_t capacity,
                     unsigned long long* plog) {
  const size_t smem = 64 * kSmallCap + 4 * (kSmallTableSlots + 33);
  if (key_words == 1) {
    cudaFuncSetAttribute(k_small_run<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_small_run<1><<<1, kSmallThreads, smem, (cudaStream_t)stream>>>(ctl, bufs, arena, pass_off,
                                                                      npasses, capacity, plog);
  } else {
    cudaFuncSetAttribute(k_small_run<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_small_run<2><<<1, kSmallThreads, smem, (cudaStream_t)stream>>>(ctl, bufs, arena, pass_off,
                                                                      npasses, capacity, plog);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace sps
