// Gather-form branching pass on the whole GPU (the insert-once rule of Sec. 3.1).
//
//   k_gather_build  every input label claims one slot of an open-addressing
//                   index table: slot = epoch (16 bits) | fingerprint (16 bits,
//                   the top of the label's hash) | index (32 bits), claimed
//                   with a 64-bit CAS. Labels are distinct, so no label
//                   comparison is needed here. A slot whose epoch differs from
//                   the pass's is free, so the table needs clearing only when
//                   the 16-bit epoch wraps. The fingerprint lets a lookup skip
//                   almost every foreign slot without reading its label.
//   k_gather_emit   every entry: inactive -> itself; active -> look up the
//                   partner label (flip mask applied); if the partner exists
//                   and this entry's selector bit is 0, the partner writes the
//                   pair; else this entry writes both outputs of the 2x2 action
//                   (each product and sum rounded once). Outputs are pruned and
//                   compacted (warp ballot, block scan, one atomic per block);
//                   the last block publishes the count and flips the buffers.
//
// No amplitude atomics: every output is computed once, so the result equals the
// scatter form bit for bit.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "sps_device.cuh"
#include "sps_internal.h"

namespace sps {
namespace {

using namespace dev;


struct GatherArgs {
  BranchOp op;
  double eps2;
  double eps;
  uint64_t capacity;
  uint64_t fail_tag;
  uint32_t load_pct, max_log2, pass_serial, epoch;
  uint32_t mg;   // label-mask buffers (MaskRing): build reads rd; emit reads rd, writes wr
  uint32_t fallback;   // 1: skip if the amplitude-only form took the pass
};

// A skipped emit still advances the label masks: the labels are those of its
// input, so buffer wr gets buffer rd's masks and rs is emptied (block 0).
// Buffer b set to masks m by the calling warp, one stripe per lane.
__device__ __forceinline__ void warp_set_label_masks(Ctl* ctl, uint32_t b, const LabelMasks& m) {
  static_assert(kMaskStripes == 32, "one stripe per lane");
  const unsigned lane = threadIdx.x & 31u;
  unsigned long long* p = ctl->lm[b][lane];
  p[0] = lane == 0 ? m.or0 : 0ull;
  p[1] = lane == 0 ? m.or1 : 0ull;
  p[2] = lane == 0 ? m.and0 : ~0ull;
  p[3] = lane == 0 ? m.and1 : ~0ull;
}

__device__ __forceinline__ void carry_label_masks(Ctl* ctl, uint32_t mg) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const LabelMasks m = read_label_masks(ctl, mg_rd(mg));
  warp_set_label_masks(ctl, mg_wr(mg), m);
  warp_set_label_masks(ctl, mg_rs(mg), LabelMasks{0ull, 0ull, ~0ull, ~0ull});
}

// The table holds n_in labels at the load factor: size for n_in, not 2 n_in.
__device__ __forceinline__ uint64_t itab_mask(uint64_t n, uint32_t load_pct, uint32_t max_log2) {
  return (1ull << table_log2_for((n + 1) / 2, load_pct, max_log2)) - 1;
}

template <int KW>
__device__ __forceinline__ void gather_build(Ctl* ctl, Bufs bufs, unsigned long long* itab,
                                             const GatherArgs& a, unsigned long long* plog) {
  const uint64_t n = ctl->nnz;
  if (plog && blockIdx.x == 0 && threadIdx.x == 0) {
    plog[0] = amp_took(ctl, a.fallback) ? 0ull : n;
    plog[1] = 0ull;
  }
  // (another block may set the status meanwhile: decide for the whole block)
  if (__syncthreads_or(ctl->status != 0u) || amp_took(ctl, a.fallback)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->index_ok = 0u;   // slots are taken over
  // Flip bits constant over the state: no entry has a partner, nothing to index.
  if (flip_bits_constant(read_label_masks_block(ctl, mg_rd(a.mg)), a.op.m)) return;
  const uint64_t mask = itab_mask(n, a.load_pct, a.max_log2);
  const SoA s = pick(bufs, ctl->cur);
  const unsigned long long ep = (unsigned long long)a.epoch << 48;
  const BranchOp& op = a.op;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k0 = s.lo[i];
    const uint64_t k1 = KW == 2 ? s.hi[i] : 0ull;
    // The partner of an active label is active too (flipping the target bits
    // keeps the controls and the Givens condition), so only active labels are
    // ever looked up: index those alone.
    bool active = (k0 & op.c[0]) == op.c[0] && (k1 & op.c[1]) == op.c[1];
    if (op.givens) active = active && (label_bit(k0, k1, op.sbit) != label_bit(k0, k1, op.qbit));
    if (!active) continue;
    const uint64_t hv = hash_label<KW>(k0, k1);
    const unsigned long long mine = ep | ((hv >> 48) << 32) | i;
    uint64_t h = hv & mask;
    bool ok = false;
    for (uint64_t p = 0; p <= mask; ++p, h = (h + 1) & mask) {
      const unsigned long long v = __ldcg(itab + h);
      if ((v & 0xFFFF000000000000ull) == ep) continue;   // taken in this pass
      if (atomicCAS(itab + h, v, mine) == v) {
        ok = true;
        break;
      }
      // lost the race: the slot now belongs to this pass, go on
    }
    if (!ok) {
      fail(ctl, SPS_ERR_TABLE_FULL, a.pass_serial, a.fail_tag);
      return;
    }
  }
}

template <int KW>
__device__ __forceinline__ uint64_t find_label(const unsigned long long* itab, uint64_t mask,
                                               unsigned long long ep, const SoA& s, uint64_t lo,
                                               uint64_t hi) {
  const uint64_t hv = hash_label<KW>(lo, hi);
  const unsigned long long fp = (hv >> 48) << 32;
  uint64_t h = hv & mask;
  for (uint64_t p = 0; p <= mask; ++p, h = (h + 1) & mask) {
    const unsigned long long v = __ldcg(itab + h);
    if ((v & 0xFFFF000000000000ull) != ep) return ~0ull;
    if ((v & 0x0000FFFF00000000ull) != fp) continue;
    const uint64_t j = v & 0xFFFFFFFFull;
    if (s.lo[j] == lo && (KW == 1 || s.hi[j] == hi)) return j;
  }
  return ~0ull;
}

template <int KW>
__device__ __forceinline__ void gather_emit(Ctl* ctl, Bufs bufs, const unsigned long long* itab,
                                            const GatherArgs& a, unsigned long long* plog) {
  __shared__ unsigned warp_cnt[32];
  __shared__ unsigned long long block_base;
  if (__syncthreads_or(ctl->status != 0u)) return;
  const uint64_t n = ctl->nnz;
  if (amp_took(ctl, a.fallback)) {
    carry_label_masks(ctl, a.mg);
    if (plog && blockIdx.x == 0 && threadIdx.x == 0) {
      plog[0] = 0ull;
      plog[1] = n;
    }
    return;
  }
  const uint64_t mask = itab_mask(n, a.load_pct, a.max_log2);
  const unsigned cur = ctl->cur;
  const SoA s = pick(bufs, cur);
  const SoA out = pick(bufs, cur ^ 1u);
  const unsigned long long ep = (unsigned long long)a.epoch << 48;
  const BranchOp& op = a.op;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned nwarps = blockDim.x >> 5;
  const bool no_partners = flip_bits_constant(read_label_masks_block(ctl, mg_rd(a.mg)), op.m);
  if (blockIdx.x == 0 && threadIdx.x == 0) reset_label_masks(ctl, mg_rs(a.mg));
  uint64_t mo0 = 0, mo1 = 0, ma0 = ~0ull, ma1 = ~0ull;   // OR / AND of the written labels
  for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x; base < n;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    uint64_t l0 = 0, h0 = 0, l1 = 0, h1 = 0;
    double v0r = 0, v0i = 0, v1r = 0, v1i = 0;
    bool w0 = false, w1 = false;
    if (i < n) {
      const uint64_t k0 = s.lo[i];
      const uint64_t k1 = KW == 2 ? s.hi[i] : 0ull;
      const double re = s.re[i], im = s.im[i];
      bool active = (k0 & op.c[0]) == op.c[0] && (k1 & op.c[1]) == op.c[1];
      const bool x = label_bit(k0, k1, op.sbit);
      if (op.givens) active = active && (x != label_bit(k0, k1, op.qbit));
      if (!active) {
        l0 = k0; h0 = k1; v0r = re; v0i = im;
        w0 = keep_amp(re, im, a.eps2, eps_pattern(a.eps));
      } else {
        const uint64_t p0 = k0 ^ op.m[0], p1 = k1 ^ op.m[1];
        const uint64_t j = no_partners ? ~0ull : find_label<KW>(itab, mask, ep, s, p0, p1);
        if (j == ~0ull || x) {   // else the partner with selector bit 1 writes the pair
          const double pre = j != ~0ull ? s.re[j] : 0.0;
          const double pim = j != ~0ull ? s.im[j] : 0.0;
          const double a0r = x ? pre : re, a0i = x ? pim : im;
          const double a1r = x ? re : pre, a1i = x ? im : pim;
          l0 = x ? p0 : k0; h0 = x ? p1 : k1;
          l1 = x ? k0 : p0; h1 = x ? k1 : p1;
          if (op.pauli)
            pair_action(pauli_pair(op, l0, h0, l1, h1), j != ~0ull, x, a0r, a0i, a1r, a1i, &v0r,
                        &v0i, &v1r, &v1i);
          else
            pair_action(op, j != ~0ull, x, a0r, a0i, a1r, a1i, &v0r, &v0i, &v1r, &v1i);
          w0 = keep_amp(v0r, v0i, a.eps2, eps_pattern(a.eps));
          w1 = keep_amp(v1r, v1i, a.eps2, eps_pattern(a.eps));
        }
      }
    }
    if (w0) {
      mo0 |= l0;
      mo1 |= h0;
      ma0 &= l0;
      ma1 &= h0;
    }
    if (w1) {
      mo0 |= l1;
      mo1 |= h1;
      ma0 &= l1;
      ma1 &= h1;
    }
    const unsigned b0 = __ballot_sync(FULL, w0), b1 = __ballot_sync(FULL, w1);
    if (lane == 0) warp_cnt[warp] = __popc(b0) + __popc(b1);
    __syncthreads();
    if (warp == 0) {
      const unsigned v = lane < nwarps ? warp_cnt[lane] : 0u;
      unsigned incl = v;
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned t = __shfl_up_sync(FULL, incl, d);
        if (lane >= (unsigned)d) incl += t;
      }
      const unsigned total = __shfl_sync(FULL, incl, 31);
      if (lane < nwarps) warp_cnt[lane] = incl - v;
      if (lane == 0)
        block_base = total ? atomicAdd(&ctl->out_count, (unsigned long long)total) : 0ull;
    }
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
    uint64_t pos = block_base + warp_cnt[warp] + __popc(b0 & below) + __popc(b1 & below);
    if (w0) {
      if (pos < a.capacity) {
        out.lo[pos] = l0;
        if (KW == 2) out.hi[pos] = h0;
        out.re[pos] = v0r;
        out.im[pos] = v0i;
      }
      ++pos;
    }
    if (w1 && pos < a.capacity) {
      out.lo[pos] = l1;
      if (KW == 2) out.hi[pos] = h1;
      out.re[pos] = v1r;
      out.im[pos] = v1i;
    }
    __syncthreads();
  }
  merge_label_masks(ctl, mg_wr(a.mg), mo0, mo1, ma0, ma1);
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&ctl->blocks_done, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      const unsigned long long total = atomicAdd(&ctl->out_count, 0ull);
      bool published = false;
      if (ctl->status == 0u) {
        if (total > a.capacity) {
          fail(ctl, SPS_ERR_CAPACITY, a.pass_serial, a.fail_tag);
        } else {
          ctl->nnz = total;
          ctl->cur = cur ^ 1u;
          ctl->updates += n;
          ctl->index_ok = 0u;   // the labels moved
          published = true;
        }
      }
      if (plog) {
        plog[0] = n;
        plog[1] = published ? total : n;
      }
      ctl->out_count = 0ull;
      ctl->blocks_done = 0u;
      __threadfence();
    }
  }
}

template <int KW>
__global__ void __launch_bounds__(256) k_gather_build(Ctl* ctl, Bufs bufs, unsigned long long* itab,
                                                      const __grid_constant__ GatherArgs a,
                                                      unsigned long long* plog) {
  gather_build<KW>(ctl, bufs, itab, a, plog);
}

// find_label for a lookup that also wants the entry's amplitude: the probe
// reads the index four slots (one 32-byte sector) at a time from the slot the
// hash names, and on a fingerprint match loads the candidate's label and
// amplitude together (the amplitude is kept if the label matches). The slots
// are scanned in the order the build claimed them, so the result is
// find_label's. Returns ~0 if the label is not indexed.
template <int KW>
__device__ __forceinline__ uint64_t find_entry(const unsigned long long* itab, uint64_t mask,
                                               unsigned long long ep, const SoA& s, uint64_t lo,
                                               uint64_t hi, double* re, double* im) {
  const uint64_t hv = hash_label<KW>(lo, hi);
  const unsigned long long fp = (hv >> 48) << 32;
  uint64_t h = hv & mask;
  uint64_t seen = 0;
  if (mask < 3) {   // a table of fewer than 4 slots: one at a time
    for (uint64_t p = 0; p <= mask; ++p, h = (h + 1) & mask) {
      const unsigned long long v = __ldcg(itab + h);
      if ((v & 0xFFFF000000000000ull) != ep) return ~0ull;
      if ((v & 0x0000FFFF00000000ull) != fp) continue;
      const uint64_t j = v & 0xFFFFFFFFull;
      if (s.lo[j] == lo && (KW == 1 || s.hi[j] == hi)) {
        *re = s.re[j];
        *im = s.im[j];
        return j;
      }
    }
    return ~0ull;
  }
  while (seen <= mask) {
    const uint64_t b = h & ~3ull;   // the table is 256-byte aligned: a 32-byte sector
    unsigned long long v4[4];
    asm("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(v4[0]), "=l"(v4[1]), "=l"(v4[2]), "=l"(v4[3])
        : "l"(itab + b));
    for (uint32_t k = (uint32_t)(h & 3ull); k < 4u; ++k) {
      const unsigned long long v = v4[k];
      ++seen;
      if ((v & 0xFFFF000000000000ull) != ep) return ~0ull;   // a free slot ends the probe
      if ((v & 0x0000FFFF00000000ull) != fp) continue;
      const uint64_t j = v & 0xFFFFFFFFull;
      const uint64_t l0 = s.lo[j];
      const uint64_t l1 = KW == 2 ? s.hi[j] : 0ull;
      const double r = s.re[j], i = s.im[j];
      if (l0 == lo && (KW == 1 || l1 == hi)) {
        *re = r;
        *im = i;
        return j;
      }
    }
    h = (b + 4) & mask;
  }
  return ~0ull;
}

template <int KW>
__global__ void __launch_bounds__(256) k_gather_emit(Ctl* ctl, Bufs bufs,
                                                     const unsigned long long* itab,
                                                     const __grid_constant__ GatherArgs a,
                                                     unsigned long long* plog) {
  gather_emit<KW>(ctl, bufs, itab, a, plog);
}

// ---------------------------------------------------------------------------
// Expansion pass (d branching gates, each active everywhere and flipping only
// qubits constant before it, so no two paths meet): output t = (i, c) with
// i = t >> d and c the d choices; label k_i ^ mask(c), amplitude a_i * F0[c0] *
// F1[c1] * F2[c2] from per-8-gate tables staged in shared memory; pruned on
// the final amplitude (every matrix entry has modulus <= 1, so no path falls
// below eps before its end and rises above it after).
// A warp owns spans of 32 E consecutive outputs, E per lane. With d >= 8 a span
// shares its input and its choices above the first 8 gates, so the warp forms
// that head once and each output costs one table product. Survivors of a span
// take one atomic for their place; the last block publishes the count.
// With WALK the phase/permutation run that follows the expansion runs on the
// outputs before they are stored (the E labels of a lane walk the op stream
// together, sharing each op's decode): the state is written once, with the
// same values as the two passes one after the other.
struct ExpandArgs {
  const double2* f;        // chunks x 256 path factors
  const ulonglong2* m;     // chunks x 256 flip masks
  uint32_t d, chunks, real, pass_serial, mg;
  double eps2, eps;
  uint64_t capacity, fail_tag;
  // the fused run that follows (WALK): op stream, fire-slot tables, gate count
  const uint4* words;
  const double2* ftab;
  uint32_t nwords, fused_gates, has_phase;
  // 1: the input is |0...0> from a reset not yet enqueued: no entry is read, and
  // the last block does the reset's work on the control block (clears the
  // status, the failure record and the update count; on a capacity failure it
  // leaves |0...0> as the state)
  uint32_t from_reset;
};

// (re, im) *= f; a real factor leaves an exactly zero imaginary part at zero
// (skipping the product, which would only give it a sign).
// Every product and sum is rounded once (see cmul_rn).
// Every lane of the warp must call it (the imaginary product of a real factor
// runs only in warps where some lane has a nonzero imaginary part: FP64 is
// scarce on this part and a predicated product still occupies the pipe).
__device__ __forceinline__ void times(bool real, double2 f, double& re, double& im) {
  if (real) {
    re = __dmul_rn(re, f.x);
    if (__any_sync(0xFFFFFFFFu, (__double_as_longlong(im) << 1) != 0)) im = __dmul_rn(im, f.x);
  } else {
    cmul_rn(re, im, f.x, f.y);
  }
}

template <int KW, int E, bool WALK>
__global__ void __launch_bounds__(256) k_expand(Ctl* ctl, Bufs bufs, const __grid_constant__ ExpandArgs a,
                                                unsigned long long* plog) {
  __shared__ double2 sf[3 * 256];
  __shared__ ulonglong2 sm[3 * 256];
  extern __shared__ uint4 fsm[];   // WALK: the op stream
  const bool rst = a.from_reset != 0u;
  if (!rst && ctl->status != 0u) return;
  const uint64_t n = rst ? 1ull : ctl->nnz;
  const unsigned cur = rst ? 0u : ctl->cur;
  const SoA s = pick(bufs, cur);
  const SoA out = pick(bufs, cur ^ 1u);
  if (blockIdx.x == 0 && threadIdx.x == 0) reset_label_masks(ctl, mg_rs(a.mg));
  for (uint32_t w = threadIdx.x; w < 256 * a.chunks; w += blockDim.x) {
    sf[w] = a.f[w];
    sm[w] = a.m[w];
  }
  if (WALK)
    for (uint32_t w = threadIdx.x; w < a.nwords; w += blockDim.x) fsm[w] = a.words[w];
  __syncthreads();
  constexpr uint32_t kSpan = 32u * E;
  const uint64_t total = n << a.d;
  const uint64_t cmask = (1ull << a.d) - 1ull;
  const uint64_t eps_bits = eps_pattern(a.eps);
  const unsigned lane = threadIdx.x & 31u;
  const bool wide = a.d >= 8;
  const uint64_t spans = (total + kSpan - 1) / kSpan;
  const uint64_t nwarp = (uint64_t)gridDim.x * (blockDim.x >> 5);
  uint64_t mo0 = 0, mo1 = 0, ma0 = ~0ull, ma1 = ~0ull;
  for (uint64_t sp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sp < spans;
       sp += nwarp) {
    const uint64_t t0 = sp * kSpan;
    uint64_t h0 = 0, h1 = 0;
    double hr = 0.0, hi = 0.0;
    if (wide) {   // the span's input and its choices above the first 8 gates
      const uint64_t i = t0 >> a.d;
      const uint32_t c = (uint32_t)(t0 & cmask);
      h0 = rst ? 0ull : s.lo[i];
      h1 = (KW == 2 && !rst) ? s.hi[i] : 0ull;
      hr = rst ? 1.0 : s.re[i];
      hi = rst ? 0.0 : s.im[i];
      for (uint32_t ch = 1; ch < a.chunks; ++ch) {
        const uint32_t u = ch * 256u + ((c >> (8u * ch)) & 0xFFu);
        h0 ^= sm[u].x;
        h1 ^= sm[u].y;
        times(a.real != 0u, sf[u], hr, hi);
      }
    }
    uint64_t L0[E], L1[E];
    double VR[E], VI[E];
    unsigned bal[E];
    unsigned count = 0;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const uint64_t t = t0 + 32u * k + lane;
      bool keep = false;
      uint64_t l0 = 0, l1 = 0;
      double vr = 0.0, vi = 0.0;
      const bool valid = t < total;
      uint32_t c0 = 0;
      if (valid) {
        if (wide) {   // a span lies inside one block of 256 choices
          c0 = (uint32_t)(t & 0xFFu);
          l0 = h0;
          l1 = h1;
          vr = hr;
          vi = hi;
        } else {
          const uint64_t i = t >> a.d;
          c0 = (uint32_t)(t & cmask);
          l0 = rst ? 0ull : s.lo[i];
          l1 = (KW == 2 && !rst) ? s.hi[i] : 0ull;
          vr = rst ? 1.0 : s.re[i];
          vi = rst ? 0.0 : s.im[i];
        }
        l0 ^= sm[c0].x;
        l1 ^= sm[c0].y;
      }
      times(a.real != 0u, sf[c0], vr, vi);   // every lane (lanes past the end on zeros)
      if (valid) keep = keep_amp(vr, vi, a.eps2, eps_bits);
      L0[k] = l0;
      L1[k] = l1;
      VR[k] = vr;
      VI[k] = vi;
      bal[k] = __ballot_sync(FULL, keep);
      count += __popc(bal[k]);
    }
    if (WALK) {   // the fused run, on every lane's E labels at once
      uint32_t cnt[E];
      uint64_t fire[E];
#pragma unroll
      for (int k = 0; k < E; ++k) {
        cnt[k] = 0u;
        fire[k] = 0ull;
      }
      walk_ops_n<KW, E>(fsm, a.nwords, L0, L1, cnt, fire);
      if (a.has_phase) {
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const uint32_t c8 = cnt[k] & 7u;
          if (((bal[k] >> lane) & 1u) && (c8 != 0u || fire[k] != 0ull)) {
            apply_fire(fire[k], a.ftab, VR[k], VI[k]);
            apply_pi4(c8, VR[k], VI[k]);
          }
        }
      }
    }
    unsigned long long base = 0ull;
    if (lane == 0 && count) base = atomicAdd(&ctl->out_count, (unsigned long long)count);
    base = __shfl_sync(FULL, base, 0);
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      if ((bal[k] >> lane) & 1u) {
        const uint64_t pos = base + __popc(bal[k] & below);
        if (pos < a.capacity) {
          out.lo[pos] = L0[k];
          if (KW == 2) out.hi[pos] = L1[k];
          out.re[pos] = VR[k];
          out.im[pos] = VI[k];
        }
        mo0 |= L0[k];
        mo1 |= L1[k];
        ma0 &= L0[k];
        ma1 &= L1[k];
      }
      base += __popc(bal[k]);
    }
  }
  merge_label_masks(ctl, mg_wr(a.mg), mo0, mo1, ma0, ma1);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&ctl->blocks_done, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      const unsigned long long got = atomicAdd(&ctl->out_count, 0ull);
      bool published = false;
      if (rst) {   // the reset's work: a clean status, no failure, no updates yet
        ctl->status = 0u;
        ctl->fail_pass = 0u;
        ctl->fail_gate = 0ull;
        ctl->updates = 0ull;
      }
      if (ctl->status == 0u) {
        if (got > a.capacity) {
          fail(ctl, SPS_ERR_CAPACITY, a.pass_serial, a.fail_tag);
          if (rst) {   // the state before the pass: |0...0> in buffer 0
            s.lo[0] = 0ull;
            if (KW == 2) s.hi[0] = 0ull;
            s.re[0] = 1.0;
            s.im[0] = 0.0;
            ctl->nnz = 1ull;
            ctl->cur = 0u;
          }
        } else {
          ctl->nnz = got;
          ctl->cur = cur ^ 1u;
          // the nonzeros before each of the d gates: n, 2n, ..., 2^(d-1) n;
          // then every gate of the fused run on the expanded state
          ctl->updates += n * cmask + got * a.fused_gates;
          published = true;
        }
      }
      if (plog) {
        plog[0] = n;
        plog[1] = published ? got : n;
      }
      ctl->out_count = 0ull;
      ctl->blocks_done = 0u;
      __threadfence();
    }
  }
}

__global__ void k_itab_clear(unsigned long long* itab, uint64_t nslots) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nslots;
       i += (uint64_t)gridDim.x * blockDim.x)
    itab[i] = 0ull;
}

// ---------------------------------------------------------------------------
// Layer pass: d <= 4 branching gates on pairwise disjoint qubits, in one
// gather pass with the same arithmetic and pruning points as d passes.
// A label k activates the gates whose controls (and Givens condition) it
// satisfies; the flips of its active gates span its group {k ^ m(S)}, and every
// member activates the same gates (no gate flips another's qubits). Members
// that differ from k only in gates with partners possible (flip qubits not
// constant, from the label masks) are looked up in the index; the present
// member with the largest selector pattern over those gates writes the group:
// it runs the gates in order over the group's amplitude vector (pair actions
// on its pairs, pruning after each gate as a pass would; an inactive gate only
// prunes) and emits the survivors. It also counts the nonzeros before each
// gate, so the update count is exact.
struct LayerArgs {
  BranchOp ops[kMaxLayerGates];
  uint32_t d;
  double eps2, eps;
  uint64_t capacity, fail_tag;
  uint32_t load_pct, max_log2, pass_serial, epoch, mg;
  uint32_t fallback;   // 1: skip if the amplitude-only form took the pass
  uint32_t force;      // amplitude-only index: rebuild whatever the device says
};

template <int KW>
__device__ __forceinline__ uint32_t layer_active(const LayerArgs& a, uint64_t k0, uint64_t k1) {
  uint32_t act = 0;
#pragma unroll
  for (uint32_t j = 0; j < kMaxLayerGates; ++j) {
    if (j < a.d) {
      const BranchOp& op = a.ops[j];
      bool on = (k0 & op.c[0]) == op.c[0] && (k1 & op.c[1]) == op.c[1];
      if (op.givens) on = on && (label_bit(k0, k1, op.sbit) != label_bit(k0, k1, op.qbit));
      act |= on ? (1u << j) : 0u;
    }
  }
  return act;
}

// Gates whose flip qubits are not constant over the state: only those can pair.
__device__ __forceinline__ uint32_t layer_pairable(const LayerArgs& a, const LabelMasks& lm) {
  uint32_t p = 0;
#pragma unroll
  for (uint32_t j = 0; j < kMaxLayerGates; ++j)
    if (j < a.d && !flip_bits_constant(lm, a.ops[j].m)) p |= 1u << j;
  return p;
}

template <int KW>
__device__ __forceinline__ void layer_build(Ctl* ctl, Bufs bufs, unsigned long long* itab,
                                            const LayerArgs& a, unsigned long long* plog) {
  const uint64_t n = ctl->nnz;
  if (plog && blockIdx.x == 0 && threadIdx.x == 0) {
    plog[0] = amp_took(ctl, a.fallback) ? 0ull : n;
    plog[1] = 0ull;
  }
  if (__syncthreads_or(ctl->status != 0u) || amp_took(ctl, a.fallback)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->index_ok = 0u;   // slots are taken over
  const uint32_t pairable = layer_pairable(a, read_label_masks_block(ctl, mg_rd(a.mg)));
  if (pairable == 0u) return;
  const uint64_t mask = itab_mask(n, a.load_pct, a.max_log2);
  const SoA s = pick(bufs, ctl->cur);
  const unsigned long long ep = (unsigned long long)a.epoch << 48;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k0 = s.lo[i];
    const uint64_t k1 = KW == 2 ? s.hi[i] : 0ull;
    if ((layer_active<KW>(a, k0, k1) & pairable) == 0u) continue;   // never looked up
    const uint64_t hv = hash_label<KW>(k0, k1);
    const unsigned long long mine = ep | ((hv >> 48) << 32) | i;
    uint64_t h = hv & mask;
    bool ok = false;
    for (uint64_t p = 0; p <= mask; ++p, h = (h + 1) & mask) {
      const unsigned long long v = __ldcg(itab + h);
      if ((v & 0xFFFF000000000000ull) == ep) continue;
      if (atomicCAS(itab + h, v, mine) == v) {
        ok = true;
        break;
      }
    }
    if (!ok) {
      fail(ctl, SPS_ERR_TABLE_FULL, a.pass_serial, a.fail_tag);
      return;
    }
  }
}

template <int KW>
__device__ __forceinline__ void layer_emit(Ctl* ctl, Bufs bufs, const unsigned long long* itab,
                                           const LayerArgs& a, unsigned long long* plog) {
  __shared__ unsigned warp_cnt[32];
  __shared__ unsigned long long block_base;
  if (__syncthreads_or(ctl->status != 0u)) return;
  const uint64_t n = ctl->nnz;
  if (amp_took(ctl, a.fallback)) {
    carry_label_masks(ctl, a.mg);
    if (plog && blockIdx.x == 0 && threadIdx.x == 0) {
      plog[0] = 0ull;
      plog[1] = n;
    }
    return;
  }
  const uint64_t mask = itab_mask(n, a.load_pct, a.max_log2);
  const unsigned cur = ctl->cur;
  const SoA s = pick(bufs, cur);
  const SoA out = pick(bufs, cur ^ 1u);
  const unsigned long long ep = (unsigned long long)a.epoch << 48;
  const uint32_t pairable = layer_pairable(a, read_label_masks_block(ctl, mg_rd(a.mg)));
  if (blockIdx.x == 0 && threadIdx.x == 0) reset_label_masks(ctl, mg_rs(a.mg));
  const uint64_t eps_bits = eps_pattern(a.eps);
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned nwarps = blockDim.x >> 5;
  uint64_t mo0 = 0, mo1 = 0, ma0 = ~0ull, ma1 = ~0ull;
  unsigned long long upd = 0;
  for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x; base < n;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    double vr[16], vi[16];
    uint32_t present = 0;   // bit u: member u of the group survives
    uint32_t act = 0;
    uint64_t k0 = 0, k1 = 0;
    uint32_t u_me = 0;
    if (i < n) {
      k0 = s.lo[i];
      k1 = KW == 2 ? s.hi[i] : 0ull;
      act = layer_active<KW>(a, k0, k1);
      // member index: bit b = the selector of the b-th active gate
      uint32_t lpos = 0;   // positions (in member-index bits) of pairable active gates
      {
        uint32_t b = 0;
#pragma unroll
        for (uint32_t j = 0; j < kMaxLayerGates; ++j) {
          if ((act >> j) & 1u) {
            if (label_bit(k0, k1, a.ops[j].sbit)) u_me |= 1u << b;
            if ((pairable >> j) & 1u) lpos |= 1u << b;
            ++b;
          }
        }
      }
      present = 1u << u_me;
      vr[u_me] = s.re[i];
      vi[u_me] = s.im[i];
      bool writer = true;
      // the other members that may be present: flips of subsets of lpos
      for (uint32_t sm = lpos; sm != 0u && writer; sm = (sm - 1u) & lpos) {
        uint64_t p0 = k0, p1 = k1;
        uint32_t b = 0;
#pragma unroll
        for (uint32_t j = 0; j < kMaxLayerGates; ++j) {
          if ((act >> j) & 1u) {
            if ((sm >> b) & 1u) {
              p0 ^= a.ops[j].m[0];
              p1 ^= a.ops[j].m[1];
            }
            ++b;
          }
        }
        const uint64_t jx = find_label<KW>(itab, mask, ep, s, p0, p1);
        if (jx == ~0ull) continue;
        const uint32_t u = u_me ^ sm;
        if ((u & lpos) > (u_me & lpos)) {
          writer = false;   // a member with a larger pattern writes the group
        } else {
          present |= 1u << u;
          vr[u] = s.re[jx];
          vi[u] = s.im[jx];
        }
      }
      if (!writer) {
        present = 0u;
      } else {
        uint32_t b = 0;
#pragma unroll
        for (uint32_t j = 0; j < kMaxLayerGates; ++j) {
          if (j < a.d) {
            upd += __popc(present);   // nonzeros of the group before gate j
            if ((act >> j) & 1u) {
              const uint32_t na = __popc(act);
              for (uint32_t u = 0; u < (1u << na); ++u) {
                if ((u >> b) & 1u) continue;
                const uint32_t u1 = u | (1u << b);
                const bool q0 = (present >> u) & 1u, q1 = (present >> u1) & 1u;
                if (!q0 && !q1) continue;
                double n0r, n0i, n1r, n1i;
                pair_action(a.ops[j], q0 && q1, q1 && !q0, q0 ? vr[u] : 0.0, q0 ? vi[u] : 0.0,
                            q1 ? vr[u1] : 0.0, q1 ? vi[u1] : 0.0, &n0r, &n0i, &n1r, &n1i);
                vr[u] = n0r;
                vi[u] = n0i;
                vr[u1] = n1r;
                vi[u1] = n1i;
                const bool w0 = keep_amp(n0r, n0i, a.eps2, eps_bits);
                const bool w1 = keep_amp(n1r, n1i, a.eps2, eps_bits);
                present = (present & ~((1u << u) | (1u << u1))) | (w0 ? 1u << u : 0u) |
                          (w1 ? 1u << u1 : 0u);
              }
              ++b;
            } else {
              for (uint32_t pr = present; pr; pr &= pr - 1u) {
                const uint32_t u = __ffs(pr) - 1u;
                if (!keep_amp(vr[u], vi[u], a.eps2, eps_bits)) present &= ~(1u << u);
              }
            }
          }
        }
      }
    }
    // compaction: each thread writes its surviving members contiguously
    const uint32_t cnt = __popc(present);
    uint32_t incl = cnt;
    for (int dd = 1; dd < 32; dd <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, incl, dd);
      if (lane >= (unsigned)dd) incl += t;
    }
    if (lane == 31) warp_cnt[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned v = lane < nwarps ? warp_cnt[lane] : 0u;
      unsigned winc = v;
      for (int dd = 1; dd < 32; dd <<= 1) {
        const unsigned t = __shfl_up_sync(FULL, winc, dd);
        if (lane >= (unsigned)dd) winc += t;
      }
      const unsigned tot = __shfl_sync(FULL, winc, 31);
      if (lane < nwarps) warp_cnt[lane] = winc - v;
      if (lane == 0) block_base = tot ? atomicAdd(&ctl->out_count, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    uint64_t pos = block_base + warp_cnt[warp] + (incl - cnt);
    for (uint32_t pr = present; pr; pr &= pr - 1u) {
      const uint32_t u = __ffs(pr) - 1u;
      uint64_t l0 = k0, l1 = k1;
      uint32_t b = 0;
#pragma unroll
      for (uint32_t j = 0; j < kMaxLayerGates; ++j) {
        if ((act >> j) & 1u) {
          if (((u ^ u_me) >> b) & 1u) {
            l0 ^= a.ops[j].m[0];
            l1 ^= a.ops[j].m[1];
          }
          ++b;
        }
      }
      if (pos < a.capacity) {
        out.lo[pos] = l0;
        if (KW == 2) out.hi[pos] = l1;
        out.re[pos] = vr[u];
        out.im[pos] = vi[u];
      }
      ++pos;
      mo0 |= l0;
      mo1 |= l1;
      ma0 &= l0;
      ma1 &= l1;
    }
    __syncthreads();
  }
  merge_label_masks(ctl, mg_wr(a.mg), mo0, mo1, ma0, ma1);
  // exact update count: the group writers' per-gate sizes
  for (int dd = 16; dd > 0; dd >>= 1) upd += __shfl_xor_sync(FULL, upd, dd);
  if (lane == 0 && upd) atomicAdd(&ctl->updates, upd);
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&ctl->blocks_done, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      const unsigned long long total = atomicAdd(&ctl->out_count, 0ull);
      bool published = false;
      if (ctl->status == 0u) {
        if (total > a.capacity) {
          fail(ctl, SPS_ERR_CAPACITY, a.pass_serial, a.fail_tag);
        } else {
          ctl->nnz = total;
          ctl->cur = cur ^ 1u;
          ctl->index_ok = 0u;   // the labels moved
          published = true;
        }
      }
      if (plog) {
        plog[0] = n;
        plog[1] = published ? total : n;
      }
      ctl->out_count = 0ull;
      ctl->blocks_done = 0u;
      __threadfence();
    }
  }
}

template <int KW>
__global__ void __launch_bounds__(256) k_layer_build(Ctl* ctl, Bufs bufs, unsigned long long* itab,
                                                     const __grid_constant__ LayerArgs a,
                                                     unsigned long long* plog) {
  layer_build<KW>(ctl, bufs, itab, a, plog);
}

template <int KW>
__global__ void __launch_bounds__(256) k_layer_emit(Ctl* ctl, Bufs bufs,
                                                    const unsigned long long* itab,
                                                    const __grid_constant__ LayerArgs a,
                                                    unsigned long long* plog) {
  layer_emit<KW>(ctl, bufs, itab, a, plog);
}

// ---------------------------------------------------------------------------
// Amplitude-only form of a run of branching passes (up to 32 gates on pairwise
// disjoint qubits). Where every active label finds each member of its group
// and no value on the way falls below eps or to zero, the run maps the set of
// labels onto itself: the state after it has the same labels, in the same
// places, with new amplitudes, and each entry is written to the same index of
// the other buffer (no compaction). A label's group is spanned by the flips of
// the gates it activates; its member with every selector bit 0 (the writer)
// takes the group: one lane looks up the partner of a pair; a group of 4, 8 or
// 16 members takes 16 lanes, one per member, that look up their members in
// parallel and run the gates in order as butterflies over shuffles (each lane
// its own row of each pair action, pruned after every gate as a pass would);
// a group of 32 or 64 takes a warp, two members per lane for 64 (the sixth
// gate pairs a lane's own two). The lookups use an index of every label that
// stays valid while passes keep labels in place. Every entry written once
// means every group had its writer; anything else (a member absent, a value
// pruned, a group of more than 64) leaves the run to the usual kernels launched after it (fallback = 1), and a
// failed attempt makes the following runs skip the attempt for a while (1, 2,
// 4 ... up to 64 runs), so states that keep changing do not pay for it.
struct AmpArgs {
  BranchOp ops[kMaxAmpGates];
  uint32_t d;
  double eps2, eps;
  uint32_t load_pct, max_log2, pass_serial, epoch, force;
  uint64_t fail_tag;
  // WALK: the phase-only fused run after the run, applied to every output
  // before it is stored (as the direct fused pass would apply it)
  const uint4* words;
  const double2* ftab;
  uint32_t nwords, fused_gates, has_phase;
  // PARITY: a phase run of signs only, as conditions (all bits set) whose
  // count of holding ones decides the sign (pi steps: 4 + 4 = a full turn)
  uint64_t par[2 * kMaxAmpParity];
  uint32_t npar;
  // 32-bit label words (bit w: label bits 32 w ..) the gates' conditions and
  // selectors read, and those the sign conditions read
  uint32_t words_act, words_par;
};

constexpr int AMP_PLAIN = 0, AMP_WALK = 1, AMP_PARITY = 2;
constexpr uint32_t kAmpMaxActive = 6;   // most active gates of a group (64 members)
#ifndef SPS_AMP_MIN_BLOCKS
#define SPS_AMP_MIN_BLOCKS 2   // resident blocks per SM the register budget allows
#endif
constexpr uint32_t kAmpRing = 64;        // per-warp queue of a size class (>= 31 + 32)

// A gate of the run as the kernel reads it, staged in shared memory: lanes
// read different gates, which from the constant bank would be serialised.
struct AmpGate {
  uint64_t c[2], m[2];
  double mre[4], mim[4];   // M[r][x] at 2 r + x
  uint32_t sbit, qbit, givens, real;
};

// 32 x 32 bit transpose over a warp: lane r passes row r (bit c = M[r][c])
// and gets column `lane` back (bit r = M[r][lane]); block swaps of 16, 8, 4,
// 2 and 1 over shuffles.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, unsigned lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const uint32_t low = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu
                       : s == 2 ? 0x33333333u : 0x55555555u;   // columns with bit s clear
    const uint32_t y = __shfl_xor_sync(FULL, x, s);
    x = (lane & s) ? ((x & ~low) | ((y >> s) & low)) : ((x & low) | ((y & low) << s));
  }
  return x;
}

// Bit-planes of the 32 labels the warp's lanes hold: pl[q] bit i = bit q of
// lane i's label, for the 32-bit label words flagged in `words` (bit w: label
// bits 32 w .. 32 w + 31). Every lane calls it.
template <int KW>
__device__ __forceinline__ void label_planes(uint32_t* pl, uint64_t k0, uint64_t k1,
                                             uint32_t words, unsigned lane) {
  __syncwarp();   // the previous planes are read
  const uint32_t w[4] = {(uint32_t)k0, (uint32_t)(k0 >> 32), (uint32_t)k1, (uint32_t)(k1 >> 32)};
#pragma unroll
  for (int q = 0; q < 2 * KW; ++q)
    if ((words >> q) & 1u) pl[32 * q + lane] = warp_transpose32(w[q], lane);
  __syncwarp();
}

// The 32 labels on which every bit of a mask (c0, c1) is set, from planes.
__device__ __forceinline__ uint32_t all_set_plane(const uint32_t* pl, uint64_t c0, uint64_t c1) {
  uint32_t A = ~0u;
  for (uint64_t m = c0; m; m &= m - 1) A &= pl[__ffsll((long long)m) - 1];
  for (uint64_t m = c1; m; m &= m - 1) A &= pl[64 + __ffsll((long long)m) - 1];
  return A;
}

// The labels that activate gate g: controls set and, for a Givens gate,
// bits p and q different.
__device__ __forceinline__ uint32_t gate_plane(const AmpGate& g, const uint32_t* pl) {
  uint32_t A = all_set_plane(pl, g.c[0], g.c[1]);
  if (g.givens) A &= pl[g.sbit] ^ pl[g.qbit];
  return A;
}

// Bit i: an odd number of the sign conditions (all bits set) hold for label
// i; lane c evaluates conditions c, c + 32 (every lane calls it).
__device__ __forceinline__ uint32_t parity_plane(const uint32_t* pl, const uint64_t* par,
                                                 uint32_t npar, unsigned lane) {
  uint32_t P = 0u;
  for (uint32_t c = lane; c < npar; c += 32) P ^= all_set_plane(pl, par[2 * c], par[2 * c + 1]);
  return __reduce_xor_sync(FULL, P);
}

// Row r of gate g's action on the pair (a0, a1) (selector bit 0, 1): M[r][0]
// a0 + M[r][1] a1 with each product and sum rounded once, as pair_action
// rounds it; REAL: every gate of the run is real (only its own products are
// issued: the FP64 pipe is scarce).
template <bool REAL>
__device__ __forceinline__ void gate_row(const AmpGate& g, int r, double a0r, double a0i,
                                         double a1r, double a1i, double* nr, double* ni) {
  const double m0 = g.mre[2 * r], m1 = g.mre[2 * r + 1];
  if (REAL || g.real) {
    *nr = __dadd_rn(__dmul_rn(m0, a0r), __dmul_rn(m1, a1r));
    *ni = __dadd_rn(__dmul_rn(m0, a0i), __dmul_rn(m1, a1i));
  } else {
    const double i0 = g.mim[2 * r], i1 = g.mim[2 * r + 1];
    const double t0r = __dsub_rn(__dmul_rn(m0, a0r), __dmul_rn(i0, a0i));
    const double t0i = __dadd_rn(__dmul_rn(m0, a0i), __dmul_rn(i0, a0r));
    const double t1r = __dsub_rn(__dmul_rn(m1, a1r), __dmul_rn(i1, a1i));
    const double t1i = __dadd_rn(__dmul_rn(m1, a1i), __dmul_rn(i1, a1r));
    *nr = __dadd_rn(t0r, t1r);
    *ni = __dadd_rn(t0i, t1i);
  }
}

// Stores one output of an amplitude-only run; POST: the phase run after it,
// walked here, or as a sign parity already decided (odd).
template <int KW, int POST>
__device__ __forceinline__ void amp_store(const AmpArgs& a, const uint4* fsm, const SoA& out,
                                          uint64_t j, uint64_t k0, uint64_t k1, double re,
                                          double im, bool odd) {
  if (POST == AMP_PARITY && odd) {   // times e^{i pi}, as apply_pi4 multiplies it
    re = -re;
    im = -im;
  }
  if (POST == AMP_WALK) {
    uint64_t l0 = k0, l1 = k1;   // a phase-only run leaves the label as it is
    uint32_t cnt = 0;
    uint64_t fire = 0ull;
    walk_ops<KW>(fsm, a.nwords, l0, l1, cnt, fire);
    cnt &= 7u;
    if (a.has_phase && (cnt != 0u || fire != 0ull)) {
      apply_fire(fire, a.ftab, re, im);
      apply_pi4(cnt, re, im);
    }
  }
  out.lo[j] = k0;
  if (KW == 2) out.hi[j] = k1;
  out.re[j] = re;
  out.im[j] = im;
}

template <int KW>
__global__ void __launch_bounds__(256) k_amp_index(Ctl* ctl, Bufs bufs, unsigned long long* itab,
                                                   const __grid_constant__ AmpArgs a,
                                                   unsigned long long* plog) {
  const bool err = ctl->status != 0u;
  const uint32_t backoff = ctl->amp_backoff;
  const bool attempt = !err && backoff == 0u;
  const bool rebuild = attempt && (a.force != 0u || ctl->index_ok == 0u);
  const uint64_t n = ctl->nnz;
  if (plog && blockIdx.x == 0 && threadIdx.x == 0) {
    plog[0] = rebuild ? n : 0ull;
    plog[1] = n;
  }
  if (rebuild) {
    const uint64_t mask = itab_mask(n, a.load_pct, a.max_log2);
    const SoA s = pick(bufs, ctl->cur);
    const unsigned long long ep = (unsigned long long)a.epoch << 48;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
      const uint64_t k0 = s.lo[i];
      const uint64_t k1 = KW == 2 ? s.hi[i] : 0ull;
      const uint64_t hv = hash_label<KW>(k0, k1);
      const unsigned long long mine = ep | ((hv >> 48) << 32) | i;
      uint64_t h = hv & mask;
      bool ok = false;
      for (uint64_t p = 0; p <= mask; ++p, h = (h + 1) & mask) {
        const unsigned long long v = __ldcg(itab + h);
        if ((v & 0xFFFF000000000000ull) == ep) continue;
        if (atomicCAS(itab + h, v, mine) == v) {
          ok = true;
          break;
        }
      }
      if (!ok) {
        fail(ctl, SPS_ERR_TABLE_FULL, a.pass_serial, a.fail_tag);
        break;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&ctl->blocks_done, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      const bool ok = ctl->status == 0u;
      if (rebuild) {
        ctl->index_ok = ok ? 1u : 0u;
        ctl->index_epoch = a.epoch;
        ctl->index_n = n;
      }
      ctl->amp_go = attempt && ok ? 1u : 0u;
      ctl->amp_state = 0u;
      ctl->amp_fail = 0u;
      ctl->out_count = 0ull;
      ctl->chunk_next = 0ull;
      if (backoff) ctl->amp_backoff = backoff - 1u;
      ctl->blocks_done = 0u;
      __threadfence();
    }
  }
}

// One round of groups of 2^c members taken from a warp's queue of writers
// (entry index, active gates): 32 >> c groups of the queue's head in aligned
// lane segments (64 members: one group, two per lane), each lane looking up
// its member and running the group's gates in order as butterflies over
// shuffles; a sign-only phase run after them is a parity, bit-sliced over
// the round's 32 labels. Every lane of the warp calls it.
template <int KW, bool REAL, int POST>
__device__ __forceinline__ void amp_round(const AmpArgs& a, const AmpGate* sg, const uint64_t* spar,
                                          uint32_t* pl, const uint4* fsm, const SoA& s,
                                          const SoA& out, const unsigned long long* itab,
                                          uint64_t mask, unsigned long long ep, uint64_t eps_bits,
                                          uint32_t c, const uint32_t* qidx, const uint32_t* qact,
                                          uint32_t head, uint32_t ng, unsigned lane, bool& bad,
                                          unsigned long long& written) {
  const uint32_t lg = c < 5u ? c : 5u;   // a group takes 2^lg lanes
  const bool two = c > 5u;               // 64 members: u and u + 32 on one lane
  const uint32_t gi = lane >> lg;
  const bool have = gi < ng;
  uint64_t wi = 0ull, w0 = 0ull, w1 = 0ull;
  uint32_t wact = 0u;
  if (have) {
    const uint32_t slot = (head + gi) % kAmpRing;
    wi = qidx[slot];
    wact = qact[slot];
    w0 = s.lo[wi];
    w1 = KW == 2 ? s.hi[wi] : 0ull;
  }
  uint32_t gidx[kAmpMaxActive];   // the group's gates, in run order
  {
    uint32_t rem = wact;
#pragma unroll
    for (uint32_t b = 0; b < kAmpMaxActive; ++b) {
      gidx[b] = rem ? (uint32_t)(__ffs(rem) - 1) : 0u;
      rem &= rem - 1u;
    }
  }
  const uint32_t u0 = lane & ((1u << lg) - 1u);
  double vr[2] = {0.0, 0.0}, vi[2] = {0.0, 0.0};
  uint64_t m0[2] = {0ull, 0ull}, m1[2] = {0ull, 0ull}, jx[2] = {~0ull, ~0ull};
  bool ok = have;
#pragma unroll
  for (uint32_t r = 0; r < 2; ++r) {
    if (!have || (r == 1 && !two)) continue;
    const uint32_t u = u0 + 32u * r;
    uint64_t l0 = w0, l1 = w1;
#pragma unroll
    for (uint32_t b = 0; b < kAmpMaxActive; ++b)
      if (b < c && ((u >> b) & 1u)) {
        const AmpGate& g = sg[gidx[b]];
        l0 ^= g.m[0];
        l1 ^= g.m[1];
      }
    m0[r] = l0;
    m1[r] = l1;
    if (u == 0u) {
      jx[r] = wi;
      vr[r] = s.re[wi];
      vi[r] = s.im[wi];
    } else {
      jx[r] = find_entry<KW>(itab, mask, ep, s, l0, l1, &vr[r], &vi[r]);
    }
    if (jx[r] == ~0ull) {
      ok = false;
    } else if ((wact & 1u) == 0u && !keep_amp(vr[r], vi[r], a.eps2, eps_bits)) {
      ok = false;   // gates before the first active one prune the inputs
    }
  }
#pragma unroll
  for (uint32_t b = 0; b < kAmpMaxActive; ++b) {
    if (b >= c) break;
    const AmpGate& g = sg[gidx[b]];
    if (b < 5u) {
      const bool x = (lane >> b) & 1u;
#pragma unroll
      for (uint32_t r = 0; r < 2; ++r) {
        if (r == 1 && !two) continue;
        const double pr = __shfl_xor_sync(FULL, vr[r], 1u << b);
        const double pi = __shfl_xor_sync(FULL, vi[r], 1u << b);
        double nr, ni;
        gate_row<REAL>(g, x ? 1 : 0, x ? pr : vr[r], x ? pi : vi[r], x ? vr[r] : pr,
                       x ? vi[r] : pi, &nr, &ni);
        vr[r] = nr;
        vi[r] = ni;
        ok = ok && keep_amp(nr, ni, a.eps2, eps_bits);
      }
    } else {   // gate 5 pairs the lane's own two members
      double n0r, n0i, n1r, n1i;
      gate_row<REAL>(g, 0, vr[0], vi[0], vr[1], vi[1], &n0r, &n0i);
      gate_row<REAL>(g, 1, vr[0], vi[0], vr[1], vi[1], &n1r, &n1i);
      vr[0] = n0r;
      vi[0] = n0i;
      vr[1] = n1r;
      vi[1] = n1i;
      ok = ok && keep_amp(n0r, n0i, a.eps2, eps_bits) && keep_amp(n1r, n1i, a.eps2, eps_bits);
    }
  }
  if (have && !ok) bad = true;
#pragma unroll
  for (uint32_t r = 0; r < 2; ++r) {
    if (r == 1 && !two) continue;
    uint32_t odd = 0u;
    if (POST == AMP_PARITY) {   // the members' signs, bit-sliced over the round
      label_planes<KW>(pl, m0[r], m1[r], a.words_par, lane);
      odd = (parity_plane(pl, spar, a.npar, lane) >> lane) & 1u;
    }
    if (have && ok) {
      amp_store<KW, POST>(a, fsm, out, jx[r], m0[r], m1[r], vr[r], vi[r], odd != 0u);
      ++written;
    }
  }
}

// One warp per chunk of 32 entries (chunks handed out by a counter), no block
// barrier inside the loop:
//   1. the chunk's labels as bit-planes in the warp's shared rows; lane j
//      evaluates gate j on all 32 (controls, Givens condition), a transpose
//      gives each entry its active gates, an OR over lanes its writer flag
//      (no active gate with the selector bit set);
//   2. entries no gate touches are copied (each gate only prunes them), with
//      the chunk's sign parity from the same planes;
//   3. writers join the warp's queue of their size class (2^c members); a
//      class runs a round (amp_round) whenever its queue holds a full one,
//      and what is left runs after the last chunk, so rounds are full.
template <int KW, bool REAL, int POST>
__global__ void __launch_bounds__(256, SPS_AMP_MIN_BLOCKS) k_amp_layer(Ctl* ctl, Bufs bufs,
                                                   const unsigned long long* itab,
                                                   const __grid_constant__ AmpArgs a,
                                                   unsigned long long* plog) {
  __shared__ AmpGate sg[kMaxAmpGates];
  __shared__ uint32_t splanes[8][128];             // per warp (<= 8 warps): label bit-planes
  __shared__ uint64_t spar[2 * kMaxAmpParity];     // sign conditions (AMP_PARITY)
  __shared__ uint32_t sqi[8][kAmpMaxActive][kAmpRing];   // per warp and class: writers' indices
  __shared__ uint32_t sqa[8][kAmpMaxActive][kAmpRing];   // and their active gates
  extern __shared__ uint4 fsm[];                   // AMP_WALK: the phase run's op stream
  const bool go = ctl->amp_go != 0u;
  if (go) {
    for (uint32_t j = threadIdx.x; j < a.d; j += blockDim.x) {
      const BranchOp& op = a.ops[j];
      AmpGate g;
      g.c[0] = op.c[0];
      g.c[1] = op.c[1];
      g.m[0] = op.m[0];
      g.m[1] = op.m[1];
      g.mre[0] = op.m_re[0][0];
      g.mre[1] = op.m_re[0][1];
      g.mre[2] = op.m_re[1][0];
      g.mre[3] = op.m_re[1][1];
      g.mim[0] = op.m_im[0][0];
      g.mim[1] = op.m_im[0][1];
      g.mim[2] = op.m_im[1][0];
      g.mim[3] = op.m_im[1][1];
      g.sbit = op.sbit;
      g.qbit = op.qbit;
      g.givens = op.givens;
      g.real = op.real_m;
      sg[j] = g;
    }
    if (POST == AMP_PARITY)
      for (uint32_t c = threadIdx.x; c < 2 * a.npar; c += blockDim.x) spar[c] = a.par[c];
    if (POST == AMP_WALK)
      for (uint32_t w = threadIdx.x; w < a.nwords; w += blockDim.x) fsm[w] = a.words[w];
  }
  __syncthreads();
  const uint64_t n = ctl->nnz;
  const unsigned cur = ctl->cur;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  bool bad = false;
  unsigned long long written = 0;   // entries this lane wrote
  if (go) {
    const uint64_t mask = itab_mask(ctl->index_n, a.load_pct, a.max_log2);
    const unsigned long long ep = (unsigned long long)ctl->index_epoch << 48;
    const SoA s = pick(bufs, cur);
    const SoA out = pick(bufs, cur ^ 1u);
    const uint64_t eps_bits = eps_pattern(a.eps);
    uint32_t* pl = splanes[warp];
    const uint32_t scan_words = a.words_act | (POST == AMP_PARITY ? a.words_par : 0u);
    uint32_t qhead[kAmpMaxActive], qtail[kAmpMaxActive];   // warp-uniform
#pragma unroll
    for (uint32_t c = 0; c < kAmpMaxActive; ++c) qhead[c] = qtail[c] = 0u;
    const uint64_t nchunks = (n + 31) / 32;
    // warps take chunks from a shared counter, so the slower ones take fewer
    // (the kernel ends with its slowest warp)
    unsigned long long ch = 0ull;
    if (lane == 0) ch = atomicAdd(&ctl->chunk_next, 1ull);
    ch = __shfl_sync(FULL, ch, 0);
    for (; ch < nchunks;) {
      unsigned long long next = 0ull;   // the next chunk is claimed before this one is worked
      if (lane == 0) next = atomicAdd(&ctl->chunk_next, 1ull);
      const uint64_t i = ch * 32 + lane;
      const bool valid = i < n;
      const uint64_t k0 = valid ? s.lo[i] : 0ull;
      const uint64_t k1 = (KW == 2 && valid) ? s.hi[i] : 0ull;
      // 1. active gates and writers
      label_planes<KW>(pl, k0, k1, scan_words, lane);
      uint32_t A = 0u, S = 0u;
      if (lane < a.d) {
        const AmpGate& g = sg[lane];
        A = gate_plane(g, pl);
        S = A & pl[g.sbit];   // active with the selector bit set: not the writer
      }
      uint32_t act = warp_transpose32(A, lane);
      const uint32_t nonwriter = __reduce_or_sync(FULL, S);
      if (!valid) act = 0u;
      const uint32_t na = __popc(act);
      const bool writer = act != 0u && !((nonwriter >> lane) & 1u);
      if (na > kAmpMaxActive) bad = true;
      // 2. entries no gate touches
      const uint32_t odd_scan = POST == AMP_PARITY ? parity_plane(pl, spar, a.npar, lane) : 0u;
      if (valid && act == 0u) {
        const double re = s.re[i], im = s.im[i];
        if (!keep_amp(re, im, a.eps2, eps_bits)) {
          bad = true;
        } else {
          amp_store<KW, POST>(a, fsm, out, i, k0, k1, re, im, (odd_scan >> lane) & 1u);
          ++written;
        }
      }
      // 3. writers into their class queues; full rounds run
#pragma unroll
      for (uint32_t c = 1; c <= kAmpMaxActive; ++c) {
        const bool mine = writer && na == c;
        const uint32_t Mc = __ballot_sync(FULL, mine);
        if (Mc == 0u) continue;
        if (mine) {
          const uint32_t slot = (qtail[c - 1] + __popc(Mc & ((1u << lane) - 1u))) % kAmpRing;
          sqi[warp][c - 1][slot] = (uint32_t)i;
          sqa[warp][c - 1][slot] = act;
        }
        qtail[c - 1] += __popc(Mc);
        __syncwarp();
        const uint32_t per = 32u >> (c < 5u ? c : 5u);   // groups per round
        while (qtail[c - 1] - qhead[c - 1] >= per) {
          amp_round<KW, REAL, POST>(a, sg, spar, pl, fsm, s, out, itab, mask, ep, eps_bits, c,
                                    sqi[warp][c - 1], sqa[warp][c - 1], qhead[c - 1], per, lane,
                                    bad, written);
          qhead[c - 1] += per;
        }
      }
      if (__any_sync(FULL, bad)) break;   // the attempt fails: the usual passes run
      ch = __shfl_sync(FULL, next, 0);
    }
    // the partial rounds left in the queues
    if (!__any_sync(FULL, bad)) {
#pragma unroll
      for (uint32_t c = 1; c <= kAmpMaxActive; ++c) {
        const uint32_t left = qtail[c - 1] - qhead[c - 1];
        if (left)
          amp_round<KW, REAL, POST>(a, sg, spar, pl, fsm, s, out, itab, mask, ep, eps_bits, c,
                                    sqi[warp][c - 1], sqa[warp][c - 1], qhead[c - 1], left, lane,
                                    bad, written);
      }
    }
    // every entry written exactly once, or some group had no writer
    for (int dd = 16; dd > 0; dd >>= 1) written += __shfl_xor_sync(FULL, written, dd);
    if (lane == 0 && written) atomicAdd(&ctl->out_count, written);
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(&ctl->amp_fail, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&ctl->blocks_done, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      const bool took = go && atomicAdd(&ctl->amp_fail, 0u) == 0u &&
                        atomicAdd(&ctl->out_count, 0ull) == n;
      if (took) {
        ctl->cur = cur ^ 1u;
        // no entry appears or goes between the gates (nor in the phase run)
        ctl->updates += n * (a.d + (POST != AMP_PLAIN ? a.fused_gates : 0u));
        ctl->amp_state = 1u;
        ctl->amp_streak = 0u;
      } else if (go) {
        const unsigned st = ctl->amp_streak;
        ctl->amp_backoff = 1u << (st < 6u ? st : 6u);
        ctl->amp_streak = st + 1u;
      }
      if (plog) {
        plog[0] = go ? n : 0ull;
        plog[1] = took ? n : 0ull;
      }
      ctl->out_count = 0ull;
      ctl->chunk_next = 0ull;
      ctl->blocks_done = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// The passes an amplitude-only attempt stands in for, in one cooperative
// launch. When the attempt took the run, block 0 carries the label masks
// through the passes' buffers (what each skipped emit does) and every block
// returns. Otherwise the passes run in order, each branching or layer pass as
// its index build, a grid barrier, its emit, and the phase-only run after them
// (walked or as a sign parity), with a grid barrier between passes. Every step
// is the body of the kernel that runs it alone, so the state equals that of
// the separate launches.
struct WalkArgs {
  const uint4* words;     // direct op stream (nwords > 0), or
  const double2* ftab;
  uint32_t nwords, has_phase;
  uint32_t npar;          // a sign parity: npar conditions (c0, c1) in par
  uint32_t ngates;        // gates of the run; 0: no run after the passes
  uint64_t par[2 * kMaxAmpParity];
};

struct ChainStep {
  uint32_t kind;   // PASS_BRANCH or PASS_LAYER
  union {
    GatherArgs g;
    LayerArgs l;
  };
};

struct ChainArgs {
  uint32_t nsteps;
  ChainStep steps[kChainSteps];
  WalkArgs w;
};
static_assert(sizeof(ChainArgs) <= 32000, "kernel parameter space");

// Barrier of every block of a cooperative launch (all resident). Thread 0
// arrives on Ctl::grid_bar (generation << 16 | broken << 15 | arrivals; the
// last arrival opens the next generation) and polls it with acquire loads. A
// wait that lasts more than a few seconds marks the barrier broken and records
// SPS_ERR_TIMEOUT; a broken barrier lets every later wait through at once, so
// the launch always ends (later steps see the status and do nothing).
constexpr uint32_t kBarrierSpins = 1u << 24;   // x ~256 ns sleep: ~4 s

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void grid_barrier(Ctl* ctl, uint32_t pass_serial, uint64_t fail_tag,
                                             uint32_t spins = kBarrierSpins) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();   // the block's writes before its arrival
    const unsigned old = atomicAdd(&ctl->grid_bar, 1u);
    if ((old & 0x7FFFu) + 1u == gridDim.x) {
      atomicAdd(&ctl->grid_bar, 0x10000u - gridDim.x);   // next generation, none arrived
    } else {
      const unsigned gen = old >> 16;
      for (uint32_t spin = 0;; ++spin) {
        const unsigned v = ld_acquire(&ctl->grid_bar);
        if ((v >> 16) != gen || (v & 0x8000u)) break;
        if (spin >= spins) {
          atomicOr(&ctl->grid_bar, 0x8000u);
          fail(ctl, SPS_ERR_TIMEOUT, pass_serial, fail_tag);
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// The phase-only run after the passes, as the direct fused pass applies it.
template <int KW>
__device__ __forceinline__ void chain_walk(Ctl* ctl, Bufs bufs, const WalkArgs& w) {
  if (ctl->status != 0u) return;
  const uint64_t n = ctl->nnz;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->updates += n * w.ngates;
  if (w.npar == 0u && (w.nwords == 0u || !w.has_phase)) return;   // labels stay: nothing to write
  const SoA s = pick(bufs, ctl->cur);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k0 = s.lo[i];
    const uint64_t k1 = KW == 2 ? s.hi[i] : 0ull;
    if (w.npar) {
      uint32_t odd = 0u;
      for (uint32_t c = 0; c < w.npar; ++c)
        odd ^= ((k0 & w.par[2 * c]) == w.par[2 * c] &&
                (k1 & w.par[2 * c + 1]) == w.par[2 * c + 1]) ? 1u : 0u;
      if (odd) {   // times e^{i pi}, as apply_pi4 multiplies it
        s.re[i] = -s.re[i];
        s.im[i] = -s.im[i];
      }
      continue;
    }
    uint64_t l0 = k0, l1 = k1;
    uint32_t cnt = 0;
    uint64_t fire = 0ull;
    walk_ops<KW>(w.words, w.nwords, l0, l1, cnt, fire);
    cnt &= 7u;
    if (cnt != 0u || fire != 0ull) {
      double re = s.re[i], im = s.im[i];
      apply_fire(fire, w.ftab, re, im);
      apply_pi4(cnt, re, im);
      s.re[i] = re;
      s.im[i] = im;
    }
  }
}

template <int KW>
__global__ void __launch_bounds__(256) k_chain(Ctl* ctl, Bufs bufs, unsigned long long* itab,
                                               const __grid_constant__ ChainArgs a,
                                               unsigned long long* plog) {
  const uint64_t n0 = ctl->nnz;
  if (amp_took(ctl, 1u)) {
    // every skipped emit copies its input's masks to its output buffer and
    // empties the next: after the chain the masks of its first input are in
    // the last step's input and output buffers, and its third buffer is empty
    if (blockIdx.x == 0 && threadIdx.x < 32 && ctl->status == 0u && a.nsteps > 0) {
      const ChainStep& s0 = a.steps[0];
      const ChainStep& sl = a.steps[a.nsteps - 1];
      const uint32_t mg0 = s0.kind == PASS_LAYER ? s0.l.mg : s0.g.mg;
      const uint32_t mgl = sl.kind == PASS_LAYER ? sl.l.mg : sl.g.mg;
      const LabelMasks m = read_label_masks(ctl, mg_rd(mg0));
      warp_set_label_masks(ctl, mg_rd(mgl), m);
      warp_set_label_masks(ctl, mg_wr(mgl), m);
      warp_set_label_masks(ctl, mg_rs(mgl), LabelMasks{0ull, 0ull, ~0ull, ~0ull});
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
      if (plog && threadIdx.x == 0) {
        plog[0] = 0ull;
        plog[1] = n0;
      }
    }
    return;
  }
  if (plog && blockIdx.x == 0 && threadIdx.x == 0) plog[0] = n0;
  uint32_t serial = 0;
  uint64_t tag = 0;
  for (uint32_t k = 0; k < a.nsteps; ++k) {
    const ChainStep& st = a.steps[k];
    serial = st.kind == PASS_LAYER ? st.l.pass_serial : st.g.pass_serial;
    tag = st.kind == PASS_LAYER ? st.l.fail_tag : st.g.fail_tag;
    if (st.kind == PASS_LAYER) {
      layer_build<KW>(ctl, bufs, itab, st.l, nullptr);
      grid_barrier(ctl, serial, tag);
      layer_emit<KW>(ctl, bufs, itab, st.l, nullptr);
    } else {
      gather_build<KW>(ctl, bufs, itab, st.g, nullptr);
      grid_barrier(ctl, serial, tag);
      gather_emit<KW>(ctl, bufs, itab, st.g, nullptr);
    }
    grid_barrier(ctl, serial, tag);
  }
  if (a.w.ngates) {
    chain_walk<KW>(ctl, bufs, a.w);
    grid_barrier(ctl, serial + 1u, tag);
  }
  if (plog && blockIdx.x == 0 && threadIdx.x == 0) plog[1] = ctl->nnz;
}

// The barrier's bounded wait, exercised: `rounds` barriers over the grid; block
// `skip` (if in the grid) does not arrive at the first one, so the others
// give up after `spins` polls and the status reads SPS_ERR_TIMEOUT.
__global__ void k_barrier_test(Ctl* ctl, uint32_t skip, uint32_t spins, uint32_t rounds) {
  for (uint32_t r = 0; r < rounds; ++r) {
    if (r == 0 && blockIdx.x == skip) continue;
    grid_barrier(ctl, r, 0ull, spins);
  }
}

int grid_of(uint64_t work, int threads, int max_blocks) {
  uint64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (uint64_t)max_blocks) b = max_blocks;
  return (int)b;
}

}  // namespace

static LayerArgs layer_args(const LayerLaunch& l, uint32_t epoch) {
  LayerArgs a;
  std::memset(&a, 0, sizeof(a));
  for (uint32_t j = 0; j < l.d; ++j) a.ops[j] = l.ops[j];
  a.d = l.d;
  a.eps2 = l.eps * l.eps;
  a.eps = l.eps;
  a.capacity = l.capacity;
  a.fail_tag = l.fail_tag;
  a.load_pct = l.load_pct;
  a.max_log2 = l.max_log2;
  a.pass_serial = l.pass_serial;
  a.epoch = epoch;
  a.mg = l.mg;
  a.fallback = l.fallback;
  return a;
}

static GatherArgs gather_args(const BranchLaunch& b, uint32_t epoch) {
  GatherArgs a;
  std::memset(&a, 0, sizeof(a));
  a.op = b.op;
  a.eps2 = b.eps * b.eps;
  a.eps = b.eps;
  a.capacity = b.capacity;
  a.fail_tag = b.fail_tag;
  a.load_pct = b.load_pct;
  a.max_log2 = b.max_log2;
  a.pass_serial = b.pass_serial;
  a.epoch = epoch;
  a.mg = b.mg;
  a.fallback = b.fallback;
  return a;
}

int launch_layer_part(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs,
                      unsigned long long* itab, uint32_t epoch, const LayerLaunch& l,
                      uint64_t nnz_bound, int part, unsigned long long* plog) {
  const LayerArgs a = layer_args(l, epoch);
  cudaStream_t st = (cudaStream_t)lc.stream;
  const int blocks = grid_of(nnz_bound, lc.threads, lc.max_blocks);
  if (part == 0) {
    if (key_words == 1)
      k_layer_build<1><<<blocks, lc.threads, 0, st>>>(ctl, bufs, itab, a, plog);
    else
      k_layer_build<2><<<blocks, lc.threads, 0, st>>>(ctl, bufs, itab, a, plog);
  } else {
    if (key_words == 1)
      k_layer_emit<1><<<blocks, lc.threads, 0, st>>>(ctl, bufs, itab, a, plog);
    else
      k_layer_emit<2><<<blocks, lc.threads, 0, st>>>(ctl, bufs, itab, a, plog);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// Resident blocks of k_chain per SM at `threads` (0 if the query fails).
template <int KW>
static int chain_blocks_per_sm(int threads) {
  static int cached[5] = {-1, -1, -1, -1, -1};   // threads 32 << k, k = 0..3
  int k = 0;
  while (k < 4 && (32 << k) < threads) ++k;
  if (cached[k] < 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_chain<KW>, threads, 0) != cudaSuccess) {
      cudaGetLastError();
      nb = 0;
    }
    cached[k] = nb;
  }
  return cached[k];
}

int launch_chain(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs,
                 unsigned long long* itab, const ChainStepDesc* steps, uint32_t nsteps,
                 const ChainWalk& w, uint64_t nnz_bound, unsigned long long* plog) {
  if (nsteps > kChainSteps || w.npar > kMaxAmpParity) return 0;
  thread_local ChainArgs a;   // ~21 KB: kept off the stack
  std::memset(&a, 0, sizeof(a));
  a.nsteps = nsteps;
  for (uint32_t k = 0; k < nsteps; ++k) {
    a.steps[k].kind = steps[k].kind;
    if (steps[k].kind == PASS_LAYER) a.steps[k].l = layer_args(steps[k].lay, steps[k].epoch);
    else a.steps[k].g = gather_args(steps[k].br, steps[k].epoch);
  }
  a.w.words = reinterpret_cast<const uint4*>(w.words);
  a.w.ftab = reinterpret_cast<const double2*>(w.ftab);
  a.w.nwords = w.nwords;
  a.w.has_phase = w.has_phase;
  a.w.npar = w.npar;
  a.w.ngates = w.ngates;
  for (uint32_t c = 0; c < 2 * w.npar; ++c) a.w.par[c] = w.par[c];
  const int threads = lc.threads < 256 ? lc.threads : 256;
  const int sms = lc.max_blocks * lc.threads / 2048;
  const int per_sm = key_words == 1 ? chain_blocks_per_sm<1>(threads) : chain_blocks_per_sm<2>(threads);
  if (per_sm <= 0 || sms <= 0) return 0;
  const int blocks = grid_of(nnz_bound, threads, per_sm * sms < 0x7FFF ? per_sm * sms : 0x7FFF);
  void* args[] = {&ctl, &bufs, &itab, &a, &plog};
  const cudaError_t e =
      key_words == 1
          ? cudaLaunchCooperativeKernel((const void*)k_chain<1>, dim3(blocks), dim3(threads), args, 0,
                                        (cudaStream_t)lc.stream)
          : cudaLaunchCooperativeKernel((const void*)k_chain<2>, dim3(blocks), dim3(threads), args, 0,
                                        (cudaStream_t)lc.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return 1;
}

// Resident blocks per SM of one k_amp_layer instance (cached per block size
// and dynamic shared memory; 0 if the query fails).
template <typename K>
static int amp_per_sm(K kern, int threads, size_t smem) {
  static int c_threads = -1, c_per = 0;
  static size_t c_smem = 0;
  if (threads != c_threads || smem != c_smem) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess) {
      cudaGetLastError();
      per = 0;
    }
    c_threads = threads;
    c_smem = smem;
    c_per = per;
  }
  return c_per;
}

// The attempt as one resident wave (each warp then works through many chunks,
// so its class queues fill whole rounds).
template <int KW, bool REAL, int POST>
static void amp_launch(int blocks, int threads, size_t smem, int sms, cudaStream_t st, Ctl* ctl,
                       Bufs bufs, const unsigned long long* itab, const AmpArgs& a,
                       unsigned long long* plog) {
  if (POST == AMP_WALK)
    cudaFuncSetAttribute(k_amp_layer<KW, REAL, POST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  const int per = amp_per_sm(k_amp_layer<KW, REAL, POST>, threads, smem);
  if (per > 0 && blocks > per * sms) blocks = per * sms;
  k_amp_layer<KW, REAL, POST><<<blocks, threads, smem, st>>>(ctl, bufs, itab, a, plog);
}

template <int KW, int POST>
static void amp_go(bool real, int blocks, int threads, size_t smem, int sms, cudaStream_t st,
                   Ctl* ctl, Bufs bufs, const unsigned long long* itab, const AmpArgs& a,
                   unsigned long long* plog) {
  if (real) amp_launch<KW, true, POST>(blocks, threads, smem, sms, st, ctl, bufs, itab, a, plog);
  else amp_launch<KW, false, POST>(blocks, threads, smem, sms, st, ctl, bufs, itab, a, plog);
}

int launch_amp_part(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs,
                    unsigned long long* itab, uint32_t epoch, uint32_t force, const AmpLaunch& l,
                    uint64_t nnz_bound, int part, unsigned long long* plog) {
  AmpArgs a;
  std::memset(&a, 0, sizeof(a));
  for (uint32_t j = 0; j < l.d; ++j) a.ops[j] = l.ops[j];
  a.d = l.d;
  a.eps2 = l.eps * l.eps;
  a.eps = l.eps;
  a.fail_tag = l.fail_tag;
  a.load_pct = l.load_pct;
  a.max_log2 = l.max_log2;
  a.pass_serial = l.pass_serial;
  a.epoch = epoch;
  a.force = force;
  a.words = reinterpret_cast<const uint4*>(l.words);
  a.ftab = reinterpret_cast<const double2*>(l.ftab);
  a.nwords = l.nwords;
  a.fused_gates = l.fused_gates;
  a.has_phase = l.has_phase;
  a.npar = l.npar;
  for (uint32_t c = 0; c < 2 * l.npar; ++c) a.par[c] = l.par[c];
  // the label words the kernel reads as bit-planes
  auto words_of = [](uint64_t lo, uint64_t hi) {
    return ((lo & 0xFFFFFFFFull) ? 1u : 0u) | ((lo >> 32) ? 2u : 0u) |
           ((hi & 0xFFFFFFFFull) ? 4u : 0u) | ((hi >> 32) ? 8u : 0u);
  };
  auto bit_words = [&](uint32_t q) {
    return words_of(q < 64 ? 1ull << q : 0ull, q >= 64 ? 1ull << (q - 64) : 0ull);
  };
  a.words_act = 0u;
  for (uint32_t j = 0; j < l.d; ++j) {
    const BranchOp& op = l.ops[j];
    a.words_act |= words_of(op.c[0], op.c[1]) | bit_words(op.sbit);
    if (op.givens) a.words_act |= bit_words(op.qbit);
  }
  a.words_par = 0u;
  for (uint32_t c = 0; c < l.npar; ++c) a.words_par |= words_of(l.par[2 * c], l.par[2 * c + 1]);
  cudaStream_t st = (cudaStream_t)lc.stream;
  const int blocks = grid_of(nnz_bound, lc.threads, lc.max_blocks);
  if (part == 0) {
    // mostly the index is still valid and the launch only decides: a quarter
    // of the resident blocks (a rebuild loops over the labels)
    const int ib = grid_of(nnz_bound, lc.threads, lc.max_blocks / 4 > 0 ? lc.max_blocks / 4 : 1);
    if (key_words == 1)
      k_amp_index<1><<<ib, lc.threads, 0, st>>>(ctl, bufs, itab, a, plog);
    else
      k_amp_index<2><<<ib, lc.threads, 0, st>>>(ctl, bufs, itab, a, plog);
  } else {
    bool real = true;
    for (uint32_t j = 0; j < l.d; ++j) real = real && l.ops[j].real_m && !l.ops[j].pauli;
    // (a phase run with no ops left only counts its gates: a walk of no words)
    const int post = l.npar ? AMP_PARITY : l.fused_gates ? AMP_WALK : AMP_PLAIN;
    const size_t smem = post == AMP_WALK ? 16 * (size_t)l.nwords : 0;
    const int sms = lc.max_blocks * lc.threads / 2048;
    if (key_words == 1) {
      if (post == AMP_PARITY) amp_go<1, AMP_PARITY>(real, blocks, lc.threads, 0, sms, st, ctl, bufs, itab, a, plog);
      else if (post == AMP_WALK) amp_go<1, AMP_WALK>(real, blocks, lc.threads, smem, sms, st, ctl, bufs, itab, a, plog);
      else amp_go<1, AMP_PLAIN>(real, blocks, lc.threads, 0, sms, st, ctl, bufs, itab, a, plog);
    } else {
      if (post == AMP_PARITY) amp_go<2, AMP_PARITY>(real, blocks, lc.threads, 0, sms, st, ctl, bufs, itab, a, plog);
      else if (post == AMP_WALK) amp_go<2, AMP_WALK>(real, blocks, lc.threads, smem, sms, st, ctl, bufs, itab, a, plog);
      else amp_go<2, AMP_PLAIN>(real, blocks, lc.threads, 0, sms, st, ctl, bufs, itab, a, plog);
    }
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_itab_clear(const LaunchCfg& lc, unsigned long long* itab, uint64_t nslots) {
  k_itab_clear<<<grid_of(nslots, lc.threads, lc.max_blocks), lc.threads, 0,
                 (cudaStream_t)lc.stream>>>(itab, nslots);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_gather_part(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs,
                       unsigned long long* itab, uint32_t epoch, const BranchLaunch& b,
                       uint64_t nnz_bound, int part, unsigned long long* plog) {
  const GatherArgs a = gather_args(b, epoch);
  cudaStream_t st = (cudaStream_t)lc.stream;
  const int blocks = grid_of(nnz_bound, lc.threads, lc.max_blocks);
  if (part == 0) {
    if (key_words == 1)
      k_gather_build<1><<<blocks, lc.threads, 0, st>>>(ctl, bufs, itab, a, plog);
    else
      k_gather_build<2><<<blocks, lc.threads, 0, st>>>(ctl, bufs, itab, a, plog);
  } else {
    if (key_words == 1)
      k_gather_emit<1><<<blocks, lc.threads, 0, st>>>(ctl, bufs, itab, a, plog);
    else
      k_gather_emit<2><<<blocks, lc.threads, 0, st>>>(ctl, bufs, itab, a, plog);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <int KW, int E, bool WALK>
static void expand_go(int blocks, int threads, size_t smem, cudaStream_t st, Ctl* ctl, Bufs bufs,
                      const ExpandArgs& a, unsigned long long* plog) {
  if (WALK)
    cudaFuncSetAttribute(k_expand<KW, E, WALK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  k_expand<KW, E, WALK><<<blocks, threads, smem, st>>>(ctl, bufs, a, plog);
}

template <int KW>
static void expand_kw(int e_log2, bool walk, int blocks, int threads, size_t smem, cudaStream_t st,
                      Ctl* ctl, Bufs bufs, const ExpandArgs& a, unsigned long long* plog) {
  if (!walk) {
    expand_go<KW, 8, false>(blocks, threads, smem, st, ctl, bufs, a, plog);
  } else if (e_log2 == 1) {
    expand_go<KW, 2, true>(blocks, threads, smem, st, ctl, bufs, a, plog);
  } else if (e_log2 == 2) {
    expand_go<KW, 4, true>(blocks, threads, smem, st, ctl, bufs, a, plog);
  } else {
    expand_go<KW, 8, true>(blocks, threads, smem, st, ctl, bufs, a, plog);
  }
}

int launch_expand(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, const ExpandLaunch& e,
                  uint64_t nnz_bound, unsigned long long* plog) {
  ExpandArgs a;
  a.f = reinterpret_cast<const double2*>(e.f);
  a.m = reinterpret_cast<const ulonglong2*>(e.m);
  a.d = e.d;
  a.chunks = (e.d + kExpandChunk - 1) / kExpandChunk;
  a.real = e.real;
  a.pass_serial = e.pass_serial;
  a.mg = e.mg;
  a.eps2 = e.eps * e.eps;
  a.eps = e.eps;
  a.capacity = e.capacity;
  a.fail_tag = e.fail_tag;
  a.words = reinterpret_cast<const uint4*>(e.words);
  a.ftab = reinterpret_cast<const double2*>(e.ftab);
  a.nwords = e.nwords;
  a.fused_gates = e.fused_gates;
  a.has_phase = e.has_phase;
  a.from_reset = e.from_reset;
  const bool walk = e.nwords > 0;
  const uint64_t total = nnz_bound << e.d;
  // Outputs per lane: 8 without a walk (measured faster than 4 on the 16.8 M
  // output expansion); with one, as many as still leave about four warps per
  // SM (more labels per lane share more decode, fewer warps hide less latency).
  int e_log2 = 3;
  if (walk) {
    // lc.max_blocks is the SM count times the resident blocks of lc.threads
    const uint64_t sms = (uint64_t)lc.max_blocks * lc.threads / 2048;
    const uint64_t warps_wanted = 4ull * (sms ? sms : 1);
    e_log2 = 1;
    while (e_log2 < 3 && total / (32ull << (e_log2 + 1)) >= warps_wanted) ++e_log2;
  }
  const uint64_t span = 32ull << e_log2;
  const uint64_t spans = (total + span - 1) / span;
  const int warps_per_block = lc.threads / 32;
  const int blocks = grid_of((spans + warps_per_block - 1) / warps_per_block * lc.threads, lc.threads,
                             lc.max_blocks);
  const size_t smem = walk ? 16 * (size_t)e.nwords : 0;
  cudaStream_t st = (cudaStream_t)lc.stream;
  if (key_words == 1)
    expand_kw<1>(e_log2, walk, blocks, lc.threads, smem, st, ctl, bufs, a, plog);
  else
    expand_kw<2>(e_log2, walk, blocks, lc.threads, smem, st, ctl, bufs, a, plog);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int barrier_selftest(uint32_t skip_block, uint32_t spins, int* status) {
  Ctl* ctl = nullptr;
  if (cudaMalloc(&ctl, sizeof(Ctl)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  int rc = -1;
  cudaStream_t st = nullptr;
  if (cudaMemset(ctl, 0, sizeof(Ctl)) == cudaSuccess &&
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) {
    uint32_t rounds = 3;
    void* args[] = {&ctl, &skip_block, &spins, &rounds};
    if (cudaLaunchCooperativeKernel((const void*)k_barrier_test, dim3(8), dim3(64), args, 0, st) ==
            cudaSuccess &&
        cudaStreamSynchronize(st) == cudaSuccess) {
      Ctl h;
      if (cudaMemcpy(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) == cudaSuccess) {
        *status = (int)h.status;
        rc = 0;
      }
    }
  }
  if (st) cudaStreamDestroy(st);
  cudaFree(ctl);
  cudaGetLastError();
  return rc;
}

}  // namespace sps
