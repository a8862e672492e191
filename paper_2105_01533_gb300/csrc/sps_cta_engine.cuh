// CTA-level pass engine (internal): one thread block applies a sequence of
// compiled passes (RunPass records) to one state. The state's two buffers and
// the index table may live in shared or global memory (generic pointers).
//
// Branching passes use the insert-once gather rule of Sec. 3.1: the block
// indexes its input labels in a table of 32-bit input indices (claimed with a
// 32-bit CAS, no amplitude atomics); every active entry looks up its partner;
// if both are present only the entry whose selector bit is 1 writes the pair,
// computing M (a0, a1) with each product and sum rounded once. Outputs are
// pruned and compacted with block scans. Fused passes run the op list per entry.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "sps_device.cuh"
#include "sps_internal.h"

namespace sps {
namespace cta {

using namespace dev;

constexpr uint32_t EMPTY_IDX = 0xFFFFFFFFu;

struct Bufs {
  uint64_t* lo;
  uint64_t* hi;   // always present (zero for 64-bit labels)
  double* re;
  double* im;
};

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
__device__ __forceinline__ uint32_t lookup(const uint32_t* tab, uint32_t mask, const Bufs& a,
                                           uint64_t lo, uint64_t hi) {
  uint32_t h = (uint32_t)hash_label<KW>(lo, hi) & mask;
  for (uint32_t p = 0; p <= mask; ++p, h = (h + 1) & mask) {
    const uint32_t j = tab[h];
    if (j == EMPTY_IDX) return EMPTY_IDX;
    if (a.lo[j] == lo && (KW == 1 || a.hi[j] == hi)) return j;
  }
  return EMPTY_IDX;
}

template <int KW>
__device__ void fused_pass(const unsigned char* arena, const RunPass& rp, const Bufs& A, uint32_t n) {
  const uint4* ops = reinterpret_cast<const uint4*>(arena + rp.ops_off);
  const double2* ftab = reinterpret_cast<const double2*>(arena + rp.ph_off);
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    uint64_t k0 = A.lo[i], k1 = A.hi[i];
    uint32_t cnt = 0;
    uint64_t fire = 0ull;
    walk_ops<KW>(ops, rp.nwords, k0, k1, cnt, fire);
    A.lo[i] = k0;
    A.hi[i] = k1;
    cnt &= 7u;
    if (cnt != 0u || fire != 0ull) {
      double re = A.re[i], im = A.im[i];
      apply_fire(fire, ftab, re, im);
      apply_pi4(cnt, re, im);
      A.re[i] = re;
      A.im[i] = im;
    }
  }
  __syncthreads();
}

// One branching pass from A (n entries) into B. Returns false, with B
// untouched beyond cap, if more than cap entries would result.
template <int KW>
__device__ bool branch_pass(const unsigned char* arena, const RunPass& rp, const Bufs& A,
                            const Bufs& B, uint32_t n, uint64_t cap, uint32_t* tab,
                            uint32_t tab_slots_max, uint32_t* warp_sums, uint32_t* n_out) {
  const BranchOp op = *reinterpret_cast<const BranchOp*>(arena + rp.br_off);
  uint32_t slots = 256;
  while (slots < 4u * n && slots < tab_slots_max) slots <<= 1;
  const uint32_t mask = slots - 1u;
  const uint64_t eps_bits = eps_pattern(rp.eps);
  for (uint32_t sl = threadIdx.x; sl < slots; sl += blockDim.x) tab[sl] = EMPTY_IDX;
  __syncthreads();
  // index the active inputs (a partner of an active label is active too)
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint64_t k0 = A.lo[i], k1 = A.hi[i];
    bool active = (k0 & op.c[0]) == op.c[0] && (k1 & op.c[1]) == op.c[1];
    if (op.givens) active = active && (label_bit(k0, k1, op.sbit) != label_bit(k0, k1, op.qbit));
    if (!active) continue;
    uint32_t h = (uint32_t)hash_label<KW>(k0, k1) & mask;
    for (uint32_t p = 0; p <= mask; ++p, h = (h + 1) & mask)
      if (atomicCAS(&tab[h], EMPTY_IDX, i) == EMPTY_IDX) break;
  }
  __syncthreads();
  uint32_t base = 0;
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
        w0 = keep_amp(re, im, rp.eps2, eps_bits);
      } else {
        const uint64_t p0 = k0 ^ op.m[0], p1 = k1 ^ op.m[1];
        const uint32_t j = lookup<KW>(tab, mask, A, p0, p1);
        if (j == EMPTY_IDX || x) {   // else the partner with selector bit 1 writes the pair
          const double pre = j != EMPTY_IDX ? A.re[j] : 0.0;
          const double pim = j != EMPTY_IDX ? A.im[j] : 0.0;
          // (a0, a1) on (label with selector 0, label with selector 1)
          const double a0r = x ? pre : re, a0i = x ? pim : im;
          const double a1r = x ? re : pre, a1i = x ? im : pim;
          l0 = x ? p0 : k0; h0 = x ? p1 : k1;
          l1 = x ? k0 : p0; h1 = x ? k1 : p1;
          if (op.pauli)
            pair_action(pauli_pair(op, l0, h0, l1, h1), j != EMPTY_IDX, x, a0r, a0i, a1r, a1i,
                        &v0r, &v0i, &v1r, &v1i);
          else
            pair_action(op, j != EMPTY_IDX, x, a0r, a0i, a1r, a1i, &v0r, &v0i, &v1r, &v1i);
          w0 = keep_amp(v0r, v0i, rp.eps2, eps_bits);
          w1 = keep_amp(v1r, v1i, rp.eps2, eps_bits);
        }
      }
    }
    uint32_t total = 0;
    const uint32_t off = base + block_scan((w0 ? 1u : 0u) + (w1 ? 1u : 0u), warp_sums, &total);
    if (base + total > cap) return false;   // uniform: every thread sees the same total
    if (w0) {
      B.lo[off] = l0; B.hi[off] = h0; B.re[off] = v0r; B.im[off] = v0i;
    }
    if (w1) {
      const uint32_t o1 = off + (w0 ? 1u : 0u);
      B.lo[o1] = l1; B.hi[o1] = h1; B.re[o1] = v1r; B.im[o1] = v1i;
    }
    base += total;
  }
  __syncthreads();
  *n_out = base;
  return true;
}

// Runs passes [p0, p1) of `passes`; A holds the n entries on entry and on exit
// (the buffers are swapped as needed). Returns the number of passes done; if
// fewer than p1 - p0, pass p0 + done failed on capacity and A still holds the
// state before it.
// *updates (nullable) accumulates, per pass done, the nonzeros before it times
// its gate count (one op per gate in a fused pass).
template <int KW>
__device__ uint32_t run_passes(const unsigned char* arena, const RunPass* passes, uint32_t p0,
                               uint32_t p1, Bufs& A, Bufs& B, uint32_t& n, uint64_t cap,
                               uint32_t* tab, uint32_t tab_slots_max, uint32_t* warp_sums,
                               uint64_t* updates = nullptr) {
  for (uint32_t pi = p0; pi < p1; ++pi) {
    const RunPass rp = passes[pi];
    if (rp.kind == PASS_FUSED) {
      fused_pass<KW>(arena, rp, A, n);
      if (updates) *updates += (uint64_t)n * rp.nops;
      continue;
    }
    if (updates) *updates += n;
    uint32_t n_out = 0;
    if (!branch_pass<KW>(arena, rp, A, B, n, cap, tab, tab_slots_max, warp_sums, &n_out)) {
      __syncthreads();
      return pi - p0;
    }
    const Bufs t = A;
    A = B;
    B = t;
    n = n_out;
  }
  return p1 - p0;
}

}  // namespace cta
}  // namespace sps
