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

// Block-wide OR/AND of per-thread label words, merged into ctl->nor/nand
// (all threads of the block must call it).
__device__ __forceinline__ void merge_label_masks(Ctl* ctl, uint64_t or0, uint64_t or1,
                                                  uint64_t and0, uint64_t and1) {
  __shared__ unsigned long long sm[4][32];
  for (int d = 16; d > 0; d >>= 1) {
    or0 |= __shfl_xor_sync(0xFFFFFFFFu, or0, d);
    or1 |= __shfl_xor_sync(0xFFFFFFFFu, or1, d);
    and0 &= __shfl_xor_sync(0xFFFFFFFFu, and0, d);
    and1 &= __shfl_xor_sync(0xFFFFFFFFu, and1, d);
  }
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sm[0][warp] = or0;
    sm[1][warp] = or1;
    sm[2][warp] = and0;
    sm[3][warp] = and1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned nw = blockDim.x >> 5;
    for (unsigned w = 1; w < nw; ++w) {
      or0 |= sm[0][w];
      or1 |= sm[1][w];
      and0 &= sm[2][w];
      and1 &= sm[3][w];
    }
    if (or0) atomicOr(&ctl->nor[0], or0);
    if (or1) atomicOr(&ctl->nor[1], or1);
    if (~and0) atomicAnd(&ctl->nand[0], and0);
    if (~and1) atomicAnd(&ctl->nand[1], and1);
  }
  __syncthreads();
}

__device__ __forceinline__ void reset_next_masks(Ctl* ctl) {
  ctl->nor[0] = ctl->nor[1] = 0ull;
  ctl->nand[0] = ctl->nand[1] = ~0ull;
}

// Publishes the next masks as current and resets them (one thread, after
// every block has merged).
__device__ __forceinline__ void publish_label_masks(Ctl* ctl) {
  ctl->cor[0] = atomicOr(&ctl->nor[0], 0ull);
  ctl->cor[1] = atomicOr(&ctl->nor[1], 0ull);
  ctl->cand[0] = atomicAnd(&ctl->nand[0], ~0ull);
  ctl->cand[1] = atomicAnd(&ctl->nand[1], ~0ull);
  reset_next_masks(ctl);
}

// Ends an in-place pass that changed labels: the last block to arrive
// publishes the merged masks.
__device__ __forceinline__ void finish_inplace_masks(Ctl* ctl) {
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&ctl->blocks_done2, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      publish_label_masks(ctl);
      ctl->blocks_done2 = 0u;
      __threadfence();
    }
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
__device__ __forceinline__ bool keep_amp(double re, double im, double eps2, uint64_t eps_bits) {
  const uint64_t ar = (uint64_t)__double_as_longlong(re) & 0x7FFFFFFFFFFFFFFFull;
  const uint64_t ai = (uint64_t)__double_as_longlong(im) & 0x7FFFFFFFFFFFFFFFull;
  if ((ar | ai) == 0ull) return false;
  if (ar >= eps_bits || ai >= eps_bits) return true;
  const double mag2 = __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
  return !(mag2 < eps2);
}

// bit pattern of eps = sqrt(eps2) as passed by the host (eps >= 0)
__device__ __forceinline__ uint64_t eps_pattern(double eps) {
  return (uint64_t)__double_as_longlong(eps);
}

}  // namespace dev
}  // namespace sps
