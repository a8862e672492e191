// Device helpers shared by the kernels of libsps (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "sps_internal.h"

namespace sps {
namespace dev {

constexpr unsigned FULL = 0xFFFFFFFFu;

struct K128 {
  uint64_t lo, hi;
};
struct __align__(16) K128a {
  uint64_t lo, hi;
};

// Buffer selection without indexing the parameter struct dynamically (which
// would copy it to local memory).
__device__ __forceinline__ SoA pick(const Bufs& b, unsigned cur) {
  SoA s;
  s.lo = cur ? b.b[1].lo : b.b[0].lo;
  s.hi = cur ? b.b[1].hi : b.b[0].hi;
  s.re = cur ? b.b[1].re : b.b[0].re;
  s.im = cur ? b.b[1].im : b.b[0].im;
  return s;
}

__device__ __forceinline__ bool label_bit(uint64_t k0, uint64_t k1, uint32_t q) {
  return q < 64 ? ((k0 >> q) & 1ull) : ((k1 >> (q - 64)) & 1ull);
}

__device__ __forceinline__ void fail(Ctl* ctl, unsigned code, uint32_t pass_serial,
                                     uint64_t fail_tag) {
  if (atomicCAS(&ctl->status, 0u, code) == 0u) {
    ctl->fail_pass = pass_serial;
    ctl->fail_gate = fail_tag;
  }
}

// ---- label masks (OR and AND of the stored labels, Ctl::lm) -------------------
struct LabelMasks { uint64_t or0, or1, and0, and1; };

// The masks in buffer b, reduced over its stripes; every lane of the calling
// warp (which must be converged) gets them.
__device__ __forceinline__ LabelMasks read_label_masks(const Ctl* ctl, uint32_t b) {
  static_assert(kMaskStripes == 32, "one stripe per lane");
  const unsigned long long* p = ctl->lm[b][threadIdx.x & 31u];
  LabelMasks m{__ldcg(p), __ldcg(p + 1), __ldcg(p + 2), __ldcg(p + 3)};
  for (int d = 16; d > 0; d >>= 1) {
    m.or0 |= __shfl_xor_sync(0xFFFFFFFFu, m.or0, d);
    m.or1 |= __shfl_xor_sync(0xFFFFFFFFu, m.or1, d);
    m.and0 &= __shfl_xor_sync(0xFFFFFFFFu, m.and0, d);
    m.and1 &= __shfl_xor_sync(0xFFFFFFFFu, m.and1, d);
  }
  return m;
}

// No entry can have a partner for a gate whose flip bits are constant over
// the state (the partner would differ in a constant bit).
__device__ __forceinline__ bool flip_bits_constant(const LabelMasks& m, const uint64_t f[2]) {
  return (((m.or0 ^ m.and0) & f[0]) | ((m.or1 ^ m.and1) & f[1])) == 0ull;
}

// Block-wide OR/AND of per-thread label words, merged into one stripe of
// buffer b with atomics whose results are not waited for (one set per block,
// so the stripes see few atomics each). Every thread of the block must call it;
// threads without labels pass (0, 0, ~0, ~0).
__device__ __forceinline__ void merge_label_masks(Ctl* ctl, uint32_t b, uint64_t or0, uint64_t or1,
                                                  uint64_t and0, uint64_t and1) {
  __shared__ unsigned long long part[4][32];
  for (int d = 16; d > 0; d >>= 1) {
    or0 |= __shfl_xor_sync(0xFFFFFFFFu, or0, d);
    or1 |= __shfl_xor_sync(0xFFFFFFFFu, or1, d);
    and0 &= __shfl_xor_sync(0xFFFFFFFFu, and0, d);
    and1 &= __shfl_xor_sync(0xFFFFFFFFu, and1, d);
  }
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (lane == 0) {
    part[0][warp] = or0;
    part[1][warp] = or1;
    part[2][warp] = and0;
    part[3][warp] = and1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (unsigned w = 1; w < (blockDim.x >> 5); ++w) {
      or0 |= part[0][w];
      or1 |= part[1][w];
      and0 &= part[2][w];
      and1 &= part[3][w];
    }
    unsigned long long* p = ctl->lm[b][blockIdx.x % kMaskStripes];
    if (or0) atomicOr(p, or0);
    if (or1) atomicOr(p + 1, or1);
    if (~and0) atomicAnd(p + 2, and0);
    if (~and1) atomicAnd(p + 3, and1);
  }
  __syncthreads();
}

// The masks in buffer b for every thread of the block (all must call it): one
// warp reads the stripes.
__device__ __forceinline__ LabelMasks read_label_masks_block(const Ctl* ctl, uint32_t b) {
  __shared__ LabelMasks shared;
  if (threadIdx.x < 32) {
    const LabelMasks m = read_label_masks(ctl, b);
    if (threadIdx.x == 0) shared = m;
  }
  __syncthreads();
  return shared;
}

// Sets buffer b to the given masks (one thread).
__device__ __forceinline__ void set_label_masks(Ctl* ctl, uint32_t b, uint64_t or0, uint64_t or1,
                                                uint64_t and0, uint64_t and1) {
  for (int i = 0; i < kMaskStripes; ++i) {
    unsigned long long* p = ctl->lm[b][i];
    p[0] = i == 0 ? or0 : 0ull;
    p[1] = i == 0 ? or1 : 0ull;
    p[2] = i == 0 ? and0 : ~0ull;
    p[3] = i == 0 ? and1 : ~0ull;
  }
}

// A fallback launch whose pass an amplitude-only attempt already produced.
__device__ __forceinline__ bool amp_took(const Ctl* ctl, uint32_t fallback) {
  return fallback != 0u && *reinterpret_cast<const volatile unsigned*>(&ctl->amp_state) == 1u;
}

// Empties buffer b for the next merge (one thread).
__device__ __forceinline__ void reset_label_masks(Ctl* ctl, uint32_t b) {
  set_label_masks(ctl, b, 0ull, 0ull, ~0ull, ~0ull);
}

// Masks that claim nothing: no qubit known constant (one thread).
__device__ __forceinline__ void unknown_label_masks(Ctl* ctl, uint32_t b) {
  set_label_masks(ctl, b, ~0ull, ~0ull, 0ull, 0ull);
}

// Runs a fused pass's encoded op stream (OPS_* runs of 16-byte words, in
// shared or global memory; every thread reads the same word, a broadcast) on
// E labels at once: flips each label in place, adds the pi/4 steps to cnt and
// sets the fire-slot bit of every arbitrary phase that applies (the product
// of those phases is taken afterwards, apply_fire). A label is handled as
// four 32-bit words, so a condition test or a flip is one three-input logic
// instruction per word.
template <int KW, int E>
__device__ __forceinline__ void walk_ops_n(const uint4* __restrict__ sq, uint32_t nwords,
                                           uint64_t (&k0)[E], uint64_t (&k1)[E],
                                           uint32_t (&cnt)[E], uint64_t (&fire)[E]) {
  uint32_t w0[E], w1[E], w2[E], w3[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    w0[e] = (uint32_t)k0[e];
    w1[e] = (uint32_t)(k0[e] >> 32);
    w2[e] = (uint32_t)k1[e];
    w3[e] = (uint32_t)(k1[e] >> 32);
  }
  uint32_t pos = 0;
  while (pos < nwords) {
    const uint4 h = sq[pos++];
    const uint32_t count = h.y;
    if (h.x == OPS_FLIP64) {
      const uint4* q = sq + pos;
#pragma unroll 8
      for (uint32_t j = 0; j < count; ++j) {
        const uint4 o = q[j];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint32_t miss = ((w0[e] & o.x) ^ o.x) | ((w1[e] & o.y) ^ o.y);
          const uint32_t m = miss == 0u ? ~0u : 0u;
          w0[e] ^= o.z & m;
          w1[e] ^= o.w & m;
        }
      }
      pos += count;
    } else if (h.x == OPS_FLIP128) {
      const uint4* q = sq + pos;
#pragma unroll 4
      for (uint32_t j = 0; j < count; ++j) {
        const uint4 c = q[2 * j], t = q[2 * j + 1];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          uint32_t miss = ((w0[e] & c.x) ^ c.x) | ((w1[e] & c.y) ^ c.y);
          if (KW == 2) miss |= ((w2[e] & c.z) ^ c.z) | ((w3[e] & c.w) ^ c.w);
          const uint32_t m = miss == 0u ? ~0u : 0u;
          w0[e] ^= t.x & m;
          w1[e] ^= t.y & m;
          if (KW == 2) {
            w2[e] ^= t.z & m;
            w3[e] ^= t.w & m;
          }
        }
      }
      pos += 2 * count;
    } else {
      const uint4* q = sq + pos;
#pragma unroll 2
      for (uint32_t j = 0; j < count; ++j) {
        const uint4 c = q[3 * j], t = q[3 * j + 1];
        const uint2 meta = *reinterpret_cast<const uint2*>(q + 3 * j + 2);
        const uint32_t kind = meta.x >> 24;   // a0 | a1 << 8 | sbit << 16 | kind << 24
        const uint32_t b = (meta.x >> 16) & 0xFFu;
        const uint32_t f0 = meta.y & 0xFFu, f1 = (meta.y >> 8) & 0xFFu;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          uint32_t miss = ((w0[e] & c.x) ^ c.x) | ((w1[e] & c.y) ^ c.y);
          if (KW == 2) miss |= ((w2[e] & c.z) ^ c.z) | ((w3[e] & c.w) ^ c.w);
          const bool cond = miss == 0u;
          bool sel = false;
          if (kind & FOP_SEL) {
            const uint32_t word = b < 32 ? w0[e] : b < 64 ? w1[e] : b < 96 ? w2[e] : w3[e];
            sel = (word >> (b & 31u)) & 1u;
          }
          cnt[e] += cond ? (sel ? (meta.x >> 8) & 0xFFu : meta.x & 0xFFu) : 0u;
          if ((kind & FOP_PH) && cond) fire[e] |= 1ull << (sel ? f1 : f0);
          const uint32_t m = cond ? ~0u : 0u;
          w0[e] ^= t.x & m;
          w1[e] ^= t.y & m;
          if (KW == 2) {
            w2[e] ^= t.z & m;
            w3[e] ^= t.w & m;
          }
        }
      }
      pos += 3 * count;
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    k0[e] = ((uint64_t)w1[e] << 32) | w0[e];
    k1[e] = ((uint64_t)w3[e] << 32) | w2[e];
  }
}

// One label at a time.
template <int KW>
__device__ __forceinline__ void walk_ops(const uint4* __restrict__ sq, uint32_t nwords,
                                         uint64_t& k0, uint64_t& k1, uint32_t& cnt,
                                         uint64_t& fire) {
  uint64_t a0[1] = {k0}, a1[1] = {k1}, f[1] = {fire};
  uint32_t c[1] = {cnt};
  walk_ops_n<KW, 1>(sq, nwords, a0, a1, c, f);
  k0 = a0[0];
  k1 = a1[0];
  cnt = c[0];
  fire = f[0];
}

// (re, im) * (tr, ti) with every product and sum rounded once (no contraction
// into fused multiply-adds), so every kernel that applies a phase gets the
// same bits whatever the compiler schedules around it.
__device__ __forceinline__ void cmul_rn(double& re, double& im, double tr, double ti) {
  const double nr = __dsub_rn(__dmul_rn(re, tr), __dmul_rn(im, ti));
  const double ni = __dadd_rn(__dmul_rn(re, ti), __dmul_rn(im, tr));
  re = nr;
  im = ni;
}

// Multiplies an amplitude by the phases of the set fire-slot bits, one table
// entry (the product of up to 8 slots' phases) per non-zero byte.
__device__ __forceinline__ void apply_fire(uint64_t fire, const double2* __restrict__ tab,
                                           double& re, double& im) {
  for (uint32_t c = 0; fire != 0ull; ++c, fire >>= 8) {
    const uint32_t v = (uint32_t)(fire & 0xFFull);
    if (v == 0u) continue;
    const double2 t = tab[c * 256u + v];
    cmul_rn(re, im, t.x, t.y);
  }
}

// Multiplies an amplitude by e^{i pi cnt / 4} (cnt mod 8), exactly for the
// quarter turns; the odd steps cost one rounding of each part.
__device__ __forceinline__ void apply_pi4(uint32_t cnt, double& re, double& im) {
  if (cnt & 1u) {  // times e^{i pi/4} = sqrt(0.5) (1 + i)
    const double r = 0.70710678118654752440;  // sqrt(0.5)
    const double nr = __dmul_rn(r, __dsub_rn(re, im));
    const double ni = __dmul_rn(r, __dadd_rn(re, im));
    re = nr;
    im = ni;
  }
  switch ((cnt >> 1) & 3u) {  // times i^(cnt/2)
    case 1: { const double t = re; re = -im; im = t; break; }
    case 2: re = -re; im = -im; break;
    case 3: { const double t = re; re = im; im = -t; break; }
    default: break;
  }
}

// murmur3 64-bit finaliser
__device__ __forceinline__ uint64_t fmix64(uint64_t z) {
  z ^= z >> 33;
  z *= 0xff51afd7ed558ccdull;
  z ^= z >> 33;
  z *= 0xc4ceb9fe1a85ec53ull;
  z ^= z >> 33;
  return z;
}

template <int KW>
__device__ __forceinline__ uint64_t hash_label(uint64_t lo, uint64_t hi) {
  if (KW == 1) return fmix64(lo);
  return fmix64(lo ^ fmix64(hi + 0x9E3779B97F4A7C15ull));
}


// contribution M[row][x] * (re, im), rounded like the plain formula
// (re*mr - im*mi, re*mi + im*mr) with every product and sum rounded once.
// (The entries are picked with selects, not a runtime index: indexing a
// kernel-parameter struct with a runtime value copies it to local memory.)
__device__ __forceinline__ void mat_times(const BranchOp& op, int row, int x, double re,
                                          double im, double* o_re, double* o_im) {
  const double mr = row == 0 ? (x ? op.m_re[0][1] : op.m_re[0][0])
                             : (x ? op.m_re[1][1] : op.m_re[1][0]);
  if (op.real_m) {
    *o_re = __dmul_rn(mr, re);
    *o_im = __dmul_rn(mr, im);
  } else {
    const double mi = row == 0 ? (x ? op.m_im[0][1] : op.m_im[0][0])
                               : (x ? op.m_im[1][1] : op.m_im[1][0]);
    *o_re = __dsub_rn(__dmul_rn(mr, re), __dmul_rn(mi, im));
    *o_im = __dadd_rn(__dmul_rn(mr, im), __dmul_rn(mi, re));
  }
}

// The 2x2 matrix of a Pauli exponential on one pair (k0: selector bit 0, k1: 1):
// P|j> = phi(j)|j ^ x> with phi(j) = i^nY (-1)^popcount(j & z), so the entry
// taking a(j) to j ^ x is -i sin(t/2) phi(j) = sin(t/2) i^(nY + 3 + 2 parity):
// a real or an imaginary +-sin, never a sum. The diagonal is cos(t/2).
__device__ __forceinline__ BranchOp pauli_pair(const BranchOp& op, uint64_t lo0, uint64_t hi0,
                                               uint64_t lo1, uint64_t hi1) {
  BranchOp m = op;
  const int e0 = (int)(op.ny + 3u + 2u * (uint32_t)(__popcll(lo0 & op.pz[0]) +
                                                    __popcll(hi0 & op.pz[1]))) & 3;
  const int e1 = (int)(op.ny + 3u + 2u * (uint32_t)(__popcll(lo1 & op.pz[0]) +
                                                    __popcll(hi1 & op.pz[1]))) & 3;
  const double sn = op.psin;
  m.m_re[1][0] = e0 == 0 ? sn : (e0 == 2 ? -sn : 0.0);   // from k0 to k1
  m.m_im[1][0] = e0 == 1 ? sn : (e0 == 3 ? -sn : 0.0);
  m.m_re[0][1] = e1 == 0 ? sn : (e1 == 2 ? -sn : 0.0);   // from k1 to k0
  m.m_im[0][1] = e1 == 1 ? sn : (e1 == 3 ? -sn : 0.0);
  m.m_im[0][0] = m.m_im[1][1] = 0.0;
  m.real_m = 0;
  return m;
}

// Both outputs of the 2x2 action on (a0, a1), the amplitudes of the labels with
// selector bit 0 and 1: n0 = M00 a0 + M01 a1, n1 = M10 a0 + M11 a1, each
// product and sum rounded once. With the partner absent one input is zero and
// its products are zeros, so n = M[.][x] a exactly (x + 0 = x; only the sign of
// a zero result can differ, and zeros are pruned).
__device__ __forceinline__ void pair_action(const BranchOp& op, bool both, bool x, double a0r,
                                            double a0i, double a1r, double a1i, double* n0r,
                                            double* n0i, double* n1r, double* n1i) {
  if (!both) {
    const int xi = x ? 1 : 0;
    const double ar = x ? a1r : a0r, ai = x ? a1i : a0i;
    mat_times(op, 0, xi, ar, ai, n0r, n0i);
    mat_times(op, 1, xi, ar, ai, n1r, n1i);
    return;
  }
  double t0r, t0i, t1r, t1i;
  mat_times(op, 0, 0, a0r, a0i, &t0r, &t0i);
  mat_times(op, 0, 1, a1r, a1i, &t1r, &t1i);
  *n0r = __dadd_rn(t0r, t1r);
  *n0i = __dadd_rn(t0i, t1i);
  mat_times(op, 1, 0, a0r, a0i, &t0r, &t0i);
  mat_times(op, 1, 1, a1r, a1i, &t1r, &t1i);
  *n1r = __dadd_rn(t0r, t1r);
  *n1i = __dadd_rn(t0i, t1i);
}

// keep an entry after a branching pass: not exactly zero and re^2 + im^2 >= eps^2
// (each product and the sum rounded once). The FP64 pipe is scarce, so the
// common cases are decided on the bit patterns: for non-negative doubles the
// IEEE order is the unsigned-integer order, and rounding is monotone, so
// |re| >= eps or |im| >= eps already implies re^2 + im^2 >= eps^2 as rounded.
// The FP64 test, out of line: inlined, the compiler evaluates it on every call
// (predicated, to avoid a branch) and the products load the scarce FP64 pipe
// although the bit-pattern tests decide almost every entry.
static __device__ __noinline__ bool keep_amp_fp64(double re, double im, double eps2) {
  const double mag2 = __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
  return !(mag2 < eps2);
}

__device__ __forceinline__ bool keep_amp(double re, double im, double eps2, uint64_t eps_bits) {
  const uint64_t ar = (uint64_t)__double_as_longlong(re) & 0x7FFFFFFFFFFFFFFFull;
  const uint64_t ai = (uint64_t)__double_as_longlong(im) & 0x7FFFFFFFFFFFFFFFull;
  if ((ar | ai) == 0ull) return false;
  if (ar >= eps_bits || ai >= eps_bits) return true;
  return keep_amp_fp64(re, im, eps2);
}

// bit pattern of eps = sqrt(eps2) as passed by the host (eps >= 0)
__device__ __forceinline__ uint64_t eps_pattern(double eps) {
  return (uint64_t)__double_as_longlong(eps);
}

}  // namespace dev
}  // namespace sps
