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
__device__ __forceinline__ void mat_times(const BranchOp& op, int row, int x, double re,
                                          double im, double* o_re, double* o_im) {
  const double mr = op.m_re[row][x];
  if (op.real_m) {
    *o_re = __dmul_rn(mr, re);
    *o_im = __dmul_rn(mr, im);
  } else {
    const double mi = op.m_im[row][x];
    *o_re = __dsub_rn(__dmul_rn(mr, re), __dmul_rn(mi, im));
    *o_im = __dadd_rn(__dmul_rn(mr, im), __dmul_rn(mi, re));
  }
}

// keep an entry after a branching pass: not exactly zero and re^2 + im^2 >= eps^2
__device__ __forceinline__ bool keep_amp(double re, double im, double eps2) {
  const double mag2 = __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
  return !(re == 0.0 && im == 0.0) && !(mag2 < eps2);
}

}  // namespace dev
}  // namespace sps
