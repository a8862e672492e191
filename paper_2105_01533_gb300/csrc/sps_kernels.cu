// CUDA kernels of libsps (sm_103a). No tensor cores: nothing on this path is a
// dense contraction. Every kernel is a grid-stride loop over a count it reads
// from the device control block, so the host never waits for a count.
//
//   k_fused          one pass per run of phase/permutation gates (Sec. 3.2):
//                    per element, run the op list on the label in registers,
//                    accumulate the phase, write back in place (a bijection
//                    keeps labels distinct, so no table is needed).
//   k_table_clear    sets table slots to EMPTY (creation and error recovery;
//                    the compaction leaves the table clean otherwise).
//   k_branch_emit    one two-nonzero gate (Sec. 3.1, Eq. 2): every element
//                    scatters its one or two contributions into an
//                    open-addressing table with 128-bit labels (claim by CAS,
//                    accumulate with FP64 atomic adds).
//   k_branch_compact walks the table, drops exact zeros and entries with
//                    re^2 + im^2 < eps^2, writes survivors to the other buffer
//                    (warp ballot + block scan + one atomic per block), cleans
//                    the slots it read and, in the last block, publishes the new
//                    count and flips the buffers.
//   k_probability    sum of |a|^2 over labels matching (mask, value) with a
//                    fixed-order two-level reduction (block sums, then the last
//                    block to finish adds them in block order).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "sps_device.cuh"
#include "sps_internal.h"

namespace sps {
namespace {

using namespace dev;

// ---------------------------------------------------------------------------
// Fused phase/permutation pass. Each block first copies the encoded op stream
// and the phases from the plan arena into shared memory (all lines in flight
// at once): walked straight from global memory, the warps of an SM advance in
// step and wait one L2 round trip for every new 128-byte line of the stream.
struct FusedArgs {
  const uint4* words;
  const double2* ftab;   // fire-slot tables (read through L1; a few entries per label)
  uint32_t nwords, ngates, has_perm, has_phase, mg;
  uint32_t fallback;     // 1: skip if an amplitude-only attempt took the pass
};

// E labels per thread (E consecutive block-wide slices of the state): the E
// labels walk the op stream together, so each op is read and decoded once for
// E labels and the E dependent chains overlap.
template <int KW, int E>
__global__ void __launch_bounds__(256) k_fused(Ctl* ctl, Bufs bufs, const FusedArgs a,
                                               unsigned long long* plog) {
  const uint64_t n = ctl->nnz;
  const bool skip = amp_took(ctl, a.fallback);
  if (plog && blockIdx.x == 0 && threadIdx.x == 0) {
    plog[0] = skip ? 0ull : n;
    plog[1] = n;
  }
  if (ctl->status != 0u || skip) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->updates += n * a.ngates;
    if (a.has_perm) reset_label_masks(ctl, mg_rs(a.mg));
  }
  const SoA s = pick(bufs, ctl->cur);
  const uint64_t slice = (uint64_t)blockDim.x;
  const uint64_t stride = (uint64_t)gridDim.x * slice * E;
  uint64_t base = blockIdx.x * slice * E + threadIdx.x;
  // the first labels are in flight while the op stream is staged
  uint64_t k0[E], k1[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint64_t i = base + e * slice;
    k0[e] = i < n ? s.lo[i] : 0ull;
    k1[e] = (KW == 2 && i < n) ? s.hi[i] : 0ull;
  }
  extern __shared__ uint4 fsm[];
  for (uint32_t w = threadIdx.x; w < a.nwords; w += blockDim.x) fsm[w] = a.words[w];
  __syncthreads();
  uint64_t mo0 = 0, mo1 = 0, ma0 = ~0ull, ma1 = ~0ull;   // OR / AND of the new labels
  for (; base < n; base += stride) {
    uint32_t cnt[E];
    uint64_t fire[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      cnt[e] = 0u;
      fire[e] = 0ull;
    }
    walk_ops_n<KW, E>(fsm, a.nwords, k0, k1, cnt, fire);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint64_t i = base + e * slice;
      if (i >= n) continue;
      if (a.has_perm) {
        s.lo[i] = k0[e];
        if (KW == 2) s.hi[i] = k1[e];
        mo0 |= k0[e];
        mo1 |= k1[e];
        ma0 &= k0[e];
        ma1 &= k1[e];
      }
      const uint32_t c8 = cnt[e] & 7u;
      if (a.has_phase && (c8 != 0u || fire[e] != 0ull)) {
        double re = s.re[i], im = s.im[i];
        apply_fire(fire[e], a.ftab, re, im);
        apply_pi4(c8, re, im);
        s.re[i] = re;
        s.im[i] = im;
      }
    }
    const uint64_t nx = base + stride;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint64_t i = nx + e * slice;
      if (i < n) {
        k0[e] = s.lo[i];
        k1[e] = KW == 2 ? s.hi[i] : 0ull;
      }
    }
  }
  if (a.has_perm) merge_label_masks(ctl, mg_wr(a.mg), mo0, mo1, ma0, ma1);
}

// ---------------------------------------------------------------------------
// Bit-sliced fused pass. A warp owns a tile of G groups x 32 entries:
//   1. load: 32 entries at a time; each 32-bit label word the pass needs is
//      transposed across the warp (shuffle butterfly), so lane j holds
//      bit-plane j of the group; planes go to shared memory, row = plane,
//      column = group (stride G + 1 keeps every access bank-conflict free);
//   2. walk: lane g runs the op list on group g's planes (one logic op handles
//      32 entries), keeping the pi/4 counter in three registers and writing
//      the fire planes of arbitrary phases to aux rows; the op list sits in
//      the kernel parameters (constant bank), so every lane reads the same op;
//   3. store: planes are transposed back; labels are written if the pass
//      permutes; each entry's aux word selects one entry per phase table, the
//      entries are multiplied in fixed point (integer pipe) and the amplitude
//      takes one FP64 complex product (two real products where it is real).

// One butterfly transpose of a 32 x 32 bit block held one word per lane:
// afterwards lane j holds bit j of every lane's word (bit i from lane i).
// Stage m exchanges m x m sub-blocks between lanes l and l ^ m: the lane keeps
// the half selected by `keep` and takes the partner's other half rotated into
// place, so a stage is a shuffle, a funnel-shift rotate and a bit select with
// per-lane constants set up once.
struct Transposer {
  uint32_t rot[5], keep[5];
  __device__ __forceinline__ void init(unsigned lane) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const uint32_t m = 16u >> i;
      const uint32_t mk = i == 0 ? 0x0000FFFFu : i == 1 ? 0x00FF00FFu : i == 2 ? 0x0F0F0F0Fu
                        : i == 3 ? 0x33333333u : 0x55555555u;
      const bool upper = (lane & m) != 0u;
      rot[i] = upper ? 32u - m : m;
      keep[i] = upper ? ~mk : mk;
    }
  }
  __device__ __forceinline__ uint32_t operator()(uint32_t x) const {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const uint32_t y = __shfl_xor_sync(FULL, x, 16u >> i);
      const uint32_t t = __funnelshift_l(y, y, rot[i]);
      x = (x & keep[i]) | (t & ~keep[i]);
    }
    return x;
  }
};

// adds the constant k (0..7) to the 3-plane counter where f is set
__device__ __forceinline__ void cnt_add(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t k,
                                        uint32_t f) {
  if (k & 1u) {
    const uint32_t carry0 = c0 & f;
    c0 ^= f;
    const uint32_t carry1 = c1 & carry0;
    c1 ^= carry0;
    c2 ^= carry1;
  }
  if (k & 2u) {
    const uint32_t carry1 = c1 & f;
    c1 ^= f;
    c2 ^= carry1;
  }
  if (k & 4u) c2 ^= f;
}

// Fixed-point complex product: a (scale 2^qa) times b (scale 2^62) gives
// scale 2^(qa - 2); three high products (a = ar + i ai, b = br + i bi):
// re = br (ar + ai) - ai (br + bi), im = br (ar + ai) + ar (bi - br).
__device__ __forceinline__ void qmul(long long& ar, long long& ai, long long br, long long bi) {
  const long long k1 = __mul64hi(br, ar + ai);
  const long long k2 = __mul64hi(ar, bi - br);
  const long long k3 = __mul64hi(ai, br + bi);
  ar = k1 - k3;
  ai = k1 + k2;
}

// v * 2^-q as a double, rounded to nearest (ties away), on the integer pipe
// (|v| >= 1 after the sign, so the result is a normal number).
__device__ __forceinline__ double q_to_double(long long v, int q) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long m = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)m);
  m <<= lz;                                     // leading one at bit 63
  unsigned long long r = (m >> 11) + ((m >> 10) & 1ull);
  int e = 63 - lz - q;
  if (r >> 53) {
    r >>= 1;
    ++e;
  }
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 1023) << 52) |
                                          (r & 0x000FFFFFFFFFFFFFull)));
}

// Op stream of the walk (kernel parameters): one 16-byte word per op,
// x, y, z = byte offsets of the three condition rows in a tile column and
// w = the target row's offset; bit 31 of w marks a general op (kind in bits
// 24..30) whose second word holds {selector row, f0 row, f1 row,
// a0 | a1 << 8}. A pure flip (X, CNOT, Toffoli) is one word; SOP_AND (the
// scratch row of long condition lists) is one word with the tag.
constexpr uint32_t kBsGeneral = 0x80000000u;

struct BsArgs {
  uint32_t nwords, ngates;
  uint32_t groups, stride;     // G, G + 1
  uint32_t rows;               // rows per tile column
  uint32_t word_bits[4];       // bits of word w that have rows
  uint32_t word_out;           // words written back
  uint32_t aux_row0, naux, ones_row;
  uint32_t has_perm, has_phase, has_cnt;
  uint32_t nchunks;
  uint32_t chunk_shift[4], chunk_bits[4];
  const longlong2* tables[4];
  const double2* direct;       // the direct phase table, or null
  uint32_t mg;                 // label-mask buffers (MaskRing)
  uint32_t fallback;           // 1: skip if an amplitude-only attempt took the pass
  uint8_t row_of[4][32];       // row of bit j of word w (kNoRow: none)
  uint4 ops[kBsMaxOps];
};

__device__ __forceinline__ uint32_t& plane(unsigned char* col, uint32_t off) {
  return *reinterpret_cast<uint32_t*>(col + off);
}

// NW: 32-bit words of a label the kernel handles (1..4); KW: 64-bit label
// words in memory (1 or 2).
template <int KW, int NW>
__global__ void __launch_bounds__(128) k_fused_bs(Ctl* ctl, Bufs bufs,
                                                  const __grid_constant__ BsArgs a,
                                                  unsigned long long* plog) {
  extern __shared__ __align__(16) uint32_t bsm[];
  const uint64_t n = ctl->nnz;
  const bool skip = amp_took(ctl, a.fallback);
  if (plog && blockIdx.x == 0 && threadIdx.x == 0) {
    plog[0] = skip ? 0ull : n;
    plog[1] = n;
  }
  if (ctl->status != 0u || skip) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->updates += n * a.ngates;
    if (a.has_perm) reset_label_masks(ctl, mg_rs(a.mg));
  }
  const SoA s = pick(bufs, ctl->cur);
  const unsigned lane = threadIdx.x & 31u;
  const unsigned warp = threadIdx.x >> 5;
  const uint32_t G = a.groups, S = a.stride;
  uint32_t* pl = bsm + (size_t)warp * a.rows * S;
  const uint64_t tile_entries = 32ull * G;
  const uint64_t ntiles = (n + tile_entries - 1) / tile_entries;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint32_t c = lane; c < S; c += 32u) pl[a.ones_row * S + c] = 0xFFFFFFFFu;
  Transposer tr;
  tr.init(lane);
  // this lane's row in each label word (offset in words; -1: none)
  int my_row[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint32_t r = a.row_of[w][lane];
    my_row[w] = r == kNoRow ? -1 : (int)(r * S);
  }
  const int aux0 = lane < a.naux ? (int)((a.aux_row0 + lane) * S) : -1;
  const int aux1 = lane + 32u < a.naux ? (int)((a.aux_row0 + 32u + lane) * S) : -1;
  uint64_t mo0 = 0, mo1 = 0, ma0 = ~0ull, ma1 = ~0ull;   // OR / AND of the new labels
  for (uint64_t tile = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile < ntiles;
       tile += nwarps) {
    const uint64_t base = tile * tile_entries;
    const uint64_t tile_n = n - base < tile_entries ? n - base : tile_entries;
    // the amplitudes are used after the walk: start moving them into L2 now
    if (a.has_phase)
      for (uint64_t off = 16ull * lane; off < tile_n; off += 512ull) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(s.re + base + off));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(s.im + base + off));
      }
    // 1. load and transpose, 8 groups at a time (their loads in flight together)
    for (uint32_t g0 = 0; g0 < G; g0 += 8u) {
      uint64_t lo[8], hi[8];
#pragma unroll
      for (uint32_t k = 0; k < 8u; ++k) {
        const uint64_t e = base + 32ull * (g0 + k) + lane;
        const bool valid = g0 + k < G && e < n;
        lo[k] = valid ? __ldcs(s.lo + e) : 0ull;
        hi[k] = (KW == 2 && valid) ? __ldcs(s.hi + e) : 0ull;
      }
#pragma unroll
      for (uint32_t k = 0; k < 8u; ++k) {
        const uint32_t g = g0 + k;
        if (g >= G) break;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          if (a.word_bits[w] == 0u) continue;
          const uint64_t src = w < 2 ? lo[k] : hi[k];
          const uint32_t t = tr((uint32_t)(src >> (32 * (w & 1))));
          if (my_row[w] >= 0) pl[my_row[w] + g] = t;
        }
      }
    }
    // the next tile's labels move into L2 while this one is walked
    {
      const uint64_t nb = base + nwarps * tile_entries;
      if (nb < n) {
        const uint64_t nn = n - nb < tile_entries ? n - nb : tile_entries;
        for (uint64_t off = 16ull * lane; off < nn; off += 512ull) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(s.lo + nb + off));
          if (KW == 2) asm volatile("prefetch.global.L2 [%0];" ::"l"(s.hi + nb + off));
        }
      }
    }
    __syncwarp();
    // 2. op walk, lane g on group g
    if (lane < G) {
      unsigned char* col = reinterpret_cast<unsigned char*>(pl + lane);
      uint32_t c0 = 0u, c1 = 0u, c2 = 0u;
      for (uint32_t j = 0; j < a.nwords;) {
        const uint4 w = a.ops[j++];
        const uint32_t f = plane(col, w.x) & plane(col, w.y) & plane(col, w.z);
        if (!(w.w & kBsGeneral)) {   // X / CNOT / Toffoli
          plane(col, w.w) ^= f;
          continue;
        }
        const uint32_t kind = (w.w >> 24) & 0x7Fu;
        const uint32_t toff = w.w & 0x00FFFFFFu;
        if (kind == SOP_AND) {
          plane(col, toff) = f;
          continue;
        }
        const uint4 e = a.ops[j++];
        const uint32_t sel = (kind & SOP_SEL) ? plane(col, e.x) : 0u;
        if (kind & SOP_CNT) {
          cnt_add(c0, c1, c2, e.w & 7u, f & ~sel);
          if (kind & SOP_SEL) cnt_add(c0, c1, c2, (e.w >> 8) & 7u, f & sel);
        }
        if (kind & SOP_FIRE) {
          plane(col, e.y) = f & ~sel;
          if (kind & SOP_SEL) plane(col, e.z) = f & sel;
        }
        if (kind & SOP_FLIP) plane(col, toff) ^= f;
      }
      if (a.has_cnt) {   // the counter planes are aux rows 0..2
        pl[a.aux_row0 * S + lane] = c0;
        pl[(a.aux_row0 + 1u) * S + lane] = c1;
        pl[(a.aux_row0 + 2u) * S + lane] = c2;
      }
    }
    __syncwarp();
    // 3. transpose back and store, 4 groups at a time: the phase-table entries
    //    and amplitudes of the 4 entries a lane writes are in flight together
    for (uint32_t g0 = 0; g0 < G; g0 += 4u) {
      uint64_t aux[4];
      uint64_t ent[4];
#pragma unroll
      for (uint32_t k = 0; k < 4u; ++k) {
        const uint32_t g = g0 + k;
        aux[k] = 0ull;
        ent[k] = base + 32ull * g + lane;
        if (g >= G) continue;
        const bool valid = ent[k] < n;
        if (a.has_perm) {
          uint64_t lo = 0ull, hi = 0ull;
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            if (!((a.word_out >> w) & 1u)) continue;
            const uint64_t x = tr(my_row[w] >= 0 ? pl[my_row[w] + g] : 0u);
            if (w < 2) lo |= x << (32 * w);
            else hi |= x << (32 * (w - 2));
          }
          if (valid) {
            if (a.word_out & 3u) s.lo[ent[k]] = lo;
            else lo = s.lo[ent[k]];
            if (KW == 2) {
              if (a.word_out & 12u) s.hi[ent[k]] = hi;
              else hi = s.hi[ent[k]];
            }
            mo0 |= lo;
            mo1 |= hi;
            ma0 &= lo;
            ma1 &= hi;
          }
        }
        if (a.has_phase) {
          const uint32_t x0 = tr(aux0 >= 0 ? pl[aux0 + g] : 0u);
          const uint32_t x1 = a.naux > 32u ? tr(aux1 >= 0 ? pl[aux1 + g] : 0u) : 0u;
          aux[k] = valid ? ((uint64_t)x0 | ((uint64_t)x1 << 32)) : 0ull;
        }
      }
      if (a.has_phase && a.direct) {   // one table of every aux pattern's phase
        double2 ph[4];
        double re[4], im[4];
#pragma unroll
        for (uint32_t k = 0; k < 4u; ++k) {
          ph[k] = make_double2(1.0, 0.0);
          re[k] = im[k] = 0.0;
          if (aux[k] == 0ull) continue;
          re[k] = __ldcs(s.re + ent[k]);
          im[k] = __ldcs(s.im + ent[k]);
          ph[k] = __ldg(a.direct + aux[k]);
        }
        // a warp whose amplitudes are all real takes two products per entry;
        // decided per warp, so the complex form is not run predicated
        bool real = true;
#pragma unroll
        for (uint32_t k = 0; k < 4u; ++k) real = real && (__double_as_longlong(im[k]) << 1) == 0;
        real = __all_sync(FULL, real);
#pragma unroll
        for (uint32_t k = 0; k < 4u; ++k) {
          if (aux[k] == 0ull) continue;
          if (real) {
            s.re[ent[k]] = re[k] * ph[k].x;
            s.im[ent[k]] = re[k] * ph[k].y;
          } else {
            s.re[ent[k]] = fma(re[k], ph[k].x, -(im[k] * ph[k].y));
            s.im[ent[k]] = fma(re[k], ph[k].y, im[k] * ph[k].x);
          }
        }
      } else if (a.has_phase) {
        const uint32_t m0 = (1u << a.chunk_bits[0]) - 1u;
        const uint32_t m1 = a.nchunks > 1 ? (1u << a.chunk_bits[1]) - 1u : 0u;
        double re[4], im[4];
        longlong2 t0[4], t1[4];
#pragma unroll
        for (uint32_t k = 0; k < 4u; ++k) {
          re[k] = im[k] = 0.0;
          t0[k] = t1[k] = make_longlong2(0, 0);
          if (aux[k] == 0ull) continue;
          re[k] = __ldcs(s.re + ent[k]);
          im[k] = __ldcs(s.im + ent[k]);
          const uint32_t i0 = (uint32_t)(aux[k] >> a.chunk_shift[0]) & m0;
          const uint32_t i1 = (uint32_t)(aux[k] >> a.chunk_shift[1]) & m1;
          if (i0) t0[k] = __ldg(a.tables[0] + i0);
          if (i1) t1[k] = __ldg(a.tables[1] + i1);
        }
#pragma unroll
        for (uint32_t k = 0; k < 4u; ++k) {
          if (aux[k] == 0ull) continue;
          long long pr = 0, pi = 0;
          int q = 62;
          bool any = false;
          if ((uint32_t)(aux[k] >> a.chunk_shift[0]) & m0) {
            pr = t0[k].x;
            pi = t0[k].y;
            any = true;
          }
          if ((uint32_t)(aux[k] >> a.chunk_shift[1]) & m1) {
            if (any) {
              qmul(pr, pi, t1[k].x, t1[k].y);
              q -= 2;
            } else {
              pr = t1[k].x;
              pi = t1[k].y;
              any = true;
            }
          }
          for (uint32_t c = 2; c < a.nchunks; ++c) {
            const uint32_t idx =
                (uint32_t)(aux[k] >> a.chunk_shift[c]) & ((1u << a.chunk_bits[c]) - 1u);
            if (idx == 0u) continue;
            const longlong2 t = __ldg(a.tables[c] + idx);
            if (any) {
              qmul(pr, pi, t.x, t.y);
              q -= 2;
            } else {
              pr = t.x;
              pi = t.y;
              any = true;
            }
          }
          const double fr = q_to_double(pr, q), fi = q_to_double(pi, q);
          if ((__double_as_longlong(im[k]) << 1) == 0) {   // a real amplitude
            s.re[ent[k]] = re[k] * fr;
            s.im[ent[k]] = re[k] * fi;
          } else {
            s.re[ent[k]] = fma(re[k], fr, -(im[k] * fi));
            s.im[ent[k]] = fma(re[k], fi, im[k] * fr);
          }
        }
      }
    }
    __syncwarp();
  }
  if (a.has_perm) merge_label_masks(ctl, mg_wr(a.mg), mo0, mo1, ma0, ma1);
}

// Phase tables of a bit-sliced pass: entry idx of chunk c is the product of
// the factors of the aux bits set in idx (fixed point, 2^62 = 1, each product
// rounded to nearest), one thread per entry.
__device__ __forceinline__ long long q62_mul(long long a, long long b) {
  const long long hi = __mul64hi(a, b);
  const unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
  // (hi:lo) >> 62, rounded: bit 61 of lo is the half
  return (long long)(((unsigned long long)hi << 2) | (lo >> 62)) + (long long)((lo >> 61) & 1ull);
}

__global__ void k_bs_tables(const longlong2* factors, longlong2* out, uint32_t bits,
                            uint32_t shift) {
  const uint32_t size = 1u << bits;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < size;
       idx += gridDim.x * blockDim.x) {
    long long re = 1ll << 62, im = 0;
    for (uint32_t m = idx; m; m &= m - 1u) {
      const longlong2 f = factors[shift + __ffs(m) - 1u];
      const long long r = q62_mul(re, f.x) - q62_mul(im, f.y);
      const long long i = q62_mul(re, f.y) + q62_mul(im, f.x);
      re = r;
      im = i;
    }
    out[idx] = make_longlong2(re, im);
  }
}

// The direct phase table: entry idx = chunk0[low bits] * chunk1[high bits]
// (fixed point, rounded once more) as doubles; with premul, times the common
// factor (c_re, c_im), in the same operations the compiled expansion applied
// to each output before (so its outputs are the same to the bit).
__global__ void k_bs_direct_table(const longlong2* c0, const longlong2* c1, uint32_t bits0,
                                  uint32_t bits, double2* out, uint32_t premul, double c_re,
                                  double c_im) {
  const uint32_t size = 1u << bits;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < size;
       idx += gridDim.x * blockDim.x) {
    const longlong2 a = c0[idx & ((1u << bits0) - 1u)];
    long long re = a.x, im = a.y;
    int q = 62;
    if (bits > bits0) {
      const longlong2 t = c1[idx >> bits0];
      qmul(re, im, t.x, t.y);
      q -= 2;
    }
    double2 v = make_double2(q_to_double(re, q), q_to_double(im, q));
    if (premul) {   // entry 0 (no phase) is the factor itself
      if (idx == 0u)
        v = make_double2(c_re, c_im);
      else if ((__double_as_longlong(c_im) << 1) == 0)
        v = make_double2(c_re * v.x, c_re * v.y);
      else
        v = make_double2(fma(c_re, v.x, -(c_im * v.y)), fma(c_re, v.y, c_im * v.x));
    }
    out[idx] = v;
  }
}

// A fused run whose gates all resolved on the host still counts its updates.
__global__ void k_count_updates(Ctl* ctl, uint32_t ngates, uint32_t fallback) {
  if (ctl->status == 0u && !amp_took(ctl, fallback)) ctl->updates += ctl->nnz * ngates;
}

// ---------------------------------------------------------------------------
__global__ void k_table_clear(Slot* table, uint64_t nslots) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nslots;
       i += (uint64_t)gridDim.x * blockDim.x) {
    ulonglong2* p = reinterpret_cast<ulonglong2*>(table + i);
    p[0] = make_ulonglong2(EMPTY, EMPTY);
    p[1] = make_ulonglong2(0ull, 0ull);
  }
}

struct BranchArgs {
  BranchOp op;
  double eps2;
  double eps;
  uint64_t capacity;
  uint64_t fail_tag;
  uint32_t load_pct, max_log2, probe_limit, pass_serial;
  uint32_t mg;   // label-mask buffers (MaskRing), for the compaction
};

// Inserts (lo, hi) -> (re, im): claims a slot for the label if it is not in
// the table yet and adds the amplitude. Returns false if `limit` slots were
// probed without finding the label or a free slot.
template <int KW>
__device__ __forceinline__ bool table_add(Slot* table, uint64_t mask, uint32_t limit,
                                          uint64_t lo, uint64_t hi, double re, double im) {
  uint64_t h = hash_label<KW>(lo, hi) & mask;
  for (uint32_t p = 0; p < limit; ++p, h = (h + 1) & mask) {
    Slot* sl = table + h;
    bool mine;
    if (KW == 1) {
      const uint64_t cur = __ldcg(&sl->lo);
      mine = cur == lo;
      if (!mine) {
        if (cur != EMPTY) continue;
        const unsigned long long old =
            atomicCAS(reinterpret_cast<unsigned long long*>(&sl->lo), EMPTY, lo);
        mine = old == EMPTY || old == lo;
        if (!mine) continue;
      }
    } else {
      // A slot changes once, from (EMPTY, EMPTY) to a label. A read that sees
      // both words different from EMPTY therefore saw a whole label (a torn read
      // has one EMPTY word); anything else is settled by the CAS.
      // A label whose low word is all ones always takes the CAS path.
      const ulonglong2 cur = __ldcg(reinterpret_cast<const ulonglong2*>(sl));
      if (cur.x != EMPTY && cur.y != EMPTY) {
        if (cur.x != lo || cur.y != hi) continue;
      } else {
        K128a expect{EMPTY, EMPTY}, want{lo, hi};
        const K128a old = atomicCAS(reinterpret_cast<K128a*>(sl), expect, want);
        mine = (old.lo == EMPTY && old.hi == EMPTY) || (old.lo == lo && old.hi == hi);
        if (!mine) continue;
      }
    }
    atomicAdd(&sl->re, re);
    atomicAdd(&sl->im, im);
    return true;
  }
  return false;
}

// The same inserts with the W lanes of a group (W = 2, 4, 8) probing W
// consecutive slots at once. The group takes its lanes' inserts in turn
// (`have`: the lane has one); for each, lane k reads slot h + k, a ballot
// finds the slots in probe order that hold the label or look free, and they
// are settled in that order: a slot with the label takes the amplitude, a free
// one is claimed by CAS (a lost race to another label moves on to the next).
// Slots only go from free to a label during the pass, so the first slot of
// the probe sequence holding the label or free is the one a single-lane probe
// would settle. Every lane of the group calls it; returns false (for the whole
// group) if an insert probed `limit` slots without a place.
template <int KW, int W>
__device__ __forceinline__ bool table_add_coop(Slot* table, uint64_t mask, uint32_t limit, bool have,
                                               uint64_t lo, uint64_t hi, double re, double im) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned sub = lane & (W - 1u);
  const unsigned base = lane - sub;
  const unsigned wm = (1u << W) - 1u;
  const unsigned gm = wm << base;   // the group's lanes
  unsigned pending = (__ballot_sync(gm, have) >> base) & wm;
  bool ok = true;
  while (pending) {
    const unsigned src = base + __ffs(pending) - 1u;
    pending &= pending - 1u;
    const uint64_t L0 = __shfl_sync(gm, lo, src);
    const uint64_t L1 = KW == 2 ? __shfl_sync(gm, hi, src) : 0ull;
    const double R = __shfl_sync(gm, re, src), I = __shfl_sync(gm, im, src);
    const uint64_t h0 = hash_label<KW>(L0, L1) & mask;
    bool done = false;
    for (uint32_t p = 0; p < limit && !done; p += W) {
      Slot* sl = table + ((h0 + p + sub) & mask);
      bool match, open;
      if (KW == 1) {
        const uint64_t cur = __ldcg(&sl->lo);
        match = cur == L0;
        open = cur == EMPTY;
      } else {
        // a read with an EMPTY word may be torn: the CAS settles it
        const ulonglong2 cur = __ldcg(reinterpret_cast<const ulonglong2*>(sl));
        open = cur.x == EMPTY || cur.y == EMPTY;
        match = !open && cur.x == L0 && cur.y == L1;
      }
      unsigned cand = (__ballot_sync(gm, p + sub < limit && (match || open)) >> base) & wm;
      while (cand) {
        const unsigned k = __ffs(cand) - 1u;
        cand &= cand - 1u;
        int got = 0;
        if (sub == k) {
          if (match) {
            got = 1;
          } else if (KW == 1) {
            const unsigned long long old =
                atomicCAS(reinterpret_cast<unsigned long long*>(&sl->lo), EMPTY, L0);
            got = old == EMPTY || old == L0;
          } else {
            K128a expect{EMPTY, EMPTY}, want{L0, L1};
            const K128a old = atomicCAS(reinterpret_cast<K128a*>(sl), expect, want);
            got = (old.lo == EMPTY && old.hi == EMPTY) || (old.lo == L0 && old.hi == L1);
          }
          if (got) {
            atomicAdd(&sl->re, R);
            atomicAdd(&sl->im, I);
          }
        }
        if (__shfl_sync(gm, got, base + k)) {
          done = true;
          break;
        }
      }
    }
    ok = ok && done;
  }
  return ok;
}

template <int KW, int W>
__global__ void __launch_bounds__(256) k_branch_emit(Ctl* ctl, Bufs bufs, Slot* table,
                                                     const __grid_constant__ BranchArgs a,
                                                     unsigned long long* plog) {
  const uint64_t n = ctl->nnz;
  if (plog && blockIdx.x == 0 && threadIdx.x == 0) {
    plog[0] = n;
    plog[1] = 0ull;
  }
  if (ctl->status != 0u) return;
  const uint64_t mask = (1ull << table_log2_for(n, a.load_pct, a.max_log2)) - 1;
  const SoA s = pick(bufs, ctl->cur);
  const BranchOp& op = a.op;
  for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x; base < n;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    // the entry's one or two contributions (label, amplitude)
    bool h0 = false, h1 = false;
    uint64_t l0 = 0, m0 = 0, l1 = 0, m1 = 0;
    double r0 = 0.0, i0 = 0.0, r1 = 0.0, i1 = 0.0;
    if (i < n) {
      const uint64_t k0 = s.lo[i];
      const uint64_t k1 = KW == 2 ? s.hi[i] : 0ull;
      const double re = s.re[i], im = s.im[i];
      bool active = (k0 & op.c[0]) == op.c[0] && (k1 & op.c[1]) == op.c[1];
      const bool x = label_bit(k0, k1, op.sbit);
      if (op.givens) active = active && (x != label_bit(k0, k1, op.qbit));
      if (!active) {
        h0 = true;
        l0 = k0;
        m0 = k1;
        r0 = re;
        i0 = im;
      } else {
        const int xi = x ? 1 : 0;
        const uint64_t f0 = k0 ^ op.m[0], f1 = k1 ^ op.m[1];
        // k0 side: the label whose selector bit is 0
        l0 = x ? f0 : k0;
        m0 = x ? f1 : k1;
        l1 = x ? k0 : f0;
        m1 = x ? k1 : f1;
        const BranchOp pm = op.pauli ? pauli_pair(op, l0, m0, l1, m1) : op;
        if (pm.m_re[0][xi] != 0.0 || pm.m_im[0][xi] != 0.0) {
          h0 = true;
          mat_times(pm, 0, xi, re, im, &r0, &i0);
        }
        if (pm.m_re[1][xi] != 0.0 || pm.m_im[1][xi] != 0.0) {
          h1 = true;
          mat_times(pm, 1, xi, re, im, &r1, &i1);
        }
      }
    }
    bool ok;
    if (W == 1) {
      ok = !h0 || table_add<KW>(table, mask, a.probe_limit, l0, m0, r0, i0);
      ok = ok && (!h1 || table_add<KW>(table, mask, a.probe_limit, l1, m1, r1, i1));
    } else {
      ok = table_add_coop<KW, W>(table, mask, a.probe_limit, h0, l0, m0, r0, i0);
      ok = table_add_coop<KW, W>(table, mask, a.probe_limit, h1, l1, m1, r1, i1) && ok;
    }
    if (!ok) {   // (W > 1: the whole group)
      fail(ctl, SPS_ERR_TABLE_FULL, a.pass_serial, a.fail_tag);
      return;
    }
  }
}

template <int KW>
__global__ void __launch_bounds__(256) k_branch_compact(Ctl* ctl, Bufs bufs, Slot* table,
                                                        const __grid_constant__ BranchArgs a,
                                                        unsigned long long* plog) {
  __shared__ unsigned warp_cnt[32];
  __shared__ unsigned long long block_base;
  const unsigned status0 = ctl->status;
  // An error from an earlier pass means this pass never filled the table.
  if (status0 != 0u && ctl->fail_pass != a.pass_serial) return;
  const bool write_ok = status0 == 0u;
  if (write_ok && blockIdx.x == 0 && threadIdx.x == 0) reset_label_masks(ctl, mg_rs(a.mg));
  const uint64_t n_in = ctl->nnz;
  const uint64_t size = 1ull << table_log2_for(n_in, a.load_pct, a.max_log2);
  const unsigned cur = ctl->cur;
  const SoA out = pick(bufs, cur ^ 1u);
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned nwarps = blockDim.x >> 5;
  uint64_t mo0 = 0, mo1 = 0, ma0 = ~0ull, ma1 = ~0ull;   // OR / AND of the kept labels
  for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x; base < size;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    bool keep = false;
    uint64_t lo = 0, hi = 0;
    double re = 0.0, im = 0.0;
    if (i < size) {
      const ulonglong2 kk = __ldcs(reinterpret_cast<const ulonglong2*>(table + i));
      const bool occ = KW == 2 ? kk.y != EMPTY : kk.x != EMPTY;
      if (occ) {
        const double2 aa = __ldcs(reinterpret_cast<const double2*>(table + i) + 1);
        lo = kk.x;
        hi = kk.y;
        re = aa.x;
        im = aa.y;
        keep = keep_amp(re, im, a.eps2, eps_pattern(a.eps));
        ulonglong2* p = reinterpret_cast<ulonglong2*>(table + i);
        p[0] = make_ulonglong2(EMPTY, EMPTY);
        p[1] = make_ulonglong2(0ull, 0ull);
      }
    }
    const unsigned ballot = __ballot_sync(FULL, keep);
    if (lane == 0) warp_cnt[warp] = __popc(ballot);
    __syncthreads();
    if (warp == 0) {
      // exclusive scan of the per-warp counts in warp 0
      unsigned v = lane < nwarps ? warp_cnt[lane] : 0u;
      unsigned incl = v;
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned t = __shfl_up_sync(FULL, incl, d);
        if (lane >= (unsigned)d) incl += t;
      }
      const unsigned total = __shfl_sync(FULL, incl, 31);
      if (lane < nwarps) warp_cnt[lane] = incl - v;
      if (lane == 0) block_base = total ? atomicAdd(&ctl->out_count, (unsigned long long)total) : 0ull;
    }
    __syncthreads();
    if (keep) {
      mo0 |= lo;
      mo1 |= hi;
      ma0 &= lo;
      ma1 &= hi;
      const uint64_t pos = block_base + warp_cnt[warp] + __popc(ballot & ((1u << lane) - 1u));
      if (write_ok && pos < a.capacity) {
        out.lo[pos] = lo;
        if (KW == 2) out.hi[pos] = hi;
        out.re[pos] = re;
        out.im[pos] = im;
      }
    }
    __syncthreads();
  }
  merge_label_masks(ctl, mg_wr(a.mg), mo0, mo1, ma0, ma1);
  // The last block to finish publishes the pass result.
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&ctl->blocks_done, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      const unsigned long long total = atomicAdd(&ctl->out_count, 0ull);
      bool published = false;
      if (write_ok) {
        if (total > a.capacity) {
          fail(ctl, SPS_ERR_CAPACITY, a.pass_serial, a.fail_tag);
        } else {
          ctl->nnz = total;
          ctl->cur = cur ^ 1u;
          ctl->updates += n_in;
          published = true;
        }
      }
      if (plog) {
        plog[0] = n_in;
        plog[1] = published ? total : n_in;
      }
      ctl->out_count = 0ull;
      ctl->blocks_done = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(FULL, v, d);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < (blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(FULL, t, d);
  }
  return t;  // valid in thread 0
}

// Each thread takes 8 consecutive entries per step (four 16-byte label loads
// in flight); a label word the mask does not test is not read at all, and
// amplitudes are read only for matching labels.
// HI: the condition reads the high label words (128-bit labels, a mask or
// value there); else only the low words are loaded.
template <int KW, bool HI>
__global__ void __launch_bounds__(256) k_probability(Ctl* ctl, Bufs bufs, uint64_t m0,
                                                     uint64_t m1, uint64_t v0, uint64_t v1,
                                                     double* partials, double* result,
                                                     unsigned long long* plog) {
  __shared__ double sh[32];
  __shared__ bool last;
  constexpr int U = HI ? 8 : 16;   // entries per lane and iteration (loads in flight)
  const uint64_t n = ctl->nnz;
  if (plog && blockIdx.x == 0 && threadIdx.x == 0) {
    plog[0] = n;
    plog[1] = n;
  }
  const SoA s = pick(bufs, ctl->cur);
  const bool use0 = (m0 | v0) != 0ull;
  constexpr bool use1 = HI;
  double acc = 0.0;
  const uint64_t stride = (uint64_t)U * gridDim.x * blockDim.x;
  // A warp reads U * 32 consecutive entries per iteration, 64 per load: load h
  // takes entries w0 + 64 h + 2 lane and the next (one contiguous 512-byte
  // span per instruction). Warps iterate together (the bound is the warp's).
  const uint64_t lane2 = 2ull * (threadIdx.x & 31u);
  for (uint64_t w0 = (uint64_t)U * (blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u));
       w0 < n; w0 += stride) {
    uint64_t k0[U], k1[U];
#pragma unroll
    for (int j = 0; j < U; ++j) k0[j] = k1[j] = 0ull;
    if (w0 + 32u * U <= n) {   // the buffers are 256-byte aligned and w0 a multiple of 256
#pragma unroll
      for (int h = 0; h < U / 2; ++h) {
        const uint64_t e = w0 + 64u * h + lane2;
        if (use0) {
          const ulonglong2 a = __ldcs(reinterpret_cast<const ulonglong2*>(s.lo + e));
          k0[2 * h] = a.x;
          k0[2 * h + 1] = a.y;
        }
        if (use1) {
          const ulonglong2 a = __ldcs(reinterpret_cast<const ulonglong2*>(s.hi + e));
          k1[2 * h] = a.x;
          k1[2 * h + 1] = a.y;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const uint64_t e = w0 + 64u * (j >> 1) + lane2 + (j & 1);
        if (e < n) {
          if (use0) k0[j] = s.lo[e];
          if (use1) k1[j] = s.hi[e];
        }
      }
    }
    uint32_t hit = 0;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const uint64_t e = w0 + 64u * (j >> 1) + lane2 + (j & 1);
      if (e < n && (k0[j] & m0) == v0 && (k1[j] & m1) == v1) hit |= 1u << j;
    }
    // FP64 is scarce on this part: only warps with a matching label run the
    // products (a predicated product still occupies the FP64 pipe)
    if (__any_sync(FULL, hit != 0u)) {
#pragma unroll
      for (int j = 0; j < U; ++j) {
        if ((hit >> j) & 1u) {
          const uint64_t e = w0 + 64u * (j >> 1) + lane2 + (j & 1);
          const double re = s.re[e], im = s.im[e];
          acc += re * re + im * im;
        }
      }
    }
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(&ctl->blocks_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s2 = 0.0;
  for (uint32_t b = threadIdx.x; b < gridDim.x; b += blockDim.x) s2 += __ldcg(partials + b);
  const double total = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    *result = total;
    ctl->blocks_done = 0u;
  }
}

// ---------------------------------------------------------------------------
// Measurement of one qubit with collapse (Sec. 2.1). k_measure_sum: block sums
// of |a|^2 over the labels with the qubit 0 and 1; the last block adds them in
// block order, draws the outcome (1 iff r * (p0 + p1) < p1) and stores
// res = {outcome, p_outcome / (p0 + p1), 1 / sqrt(p_outcome)}. k_collapse keeps
// the labels that show the outcome, scales them and compacts them into the
// other buffer; its last block publishes the count.
template <int KW>
__global__ void __launch_bounds__(256) k_measure_sum(Ctl* ctl, Bufs bufs, uint32_t word,
                                                     uint64_t bit, double r, double* partials,
                                                     double* res) {
  __shared__ double sh[32];
  __shared__ bool last;
  if (ctl->status != 0u) return;
  const uint64_t n = ctl->nnz;
  const SoA s = pick(bufs, ctl->cur);
  double a0 = 0.0, a1 = 0.0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = (KW == 2 && word) ? s.hi[i] : s.lo[i];
    const double re = s.re[i], im = s.im[i];
    const double m = re * re + im * im;
    if (k & bit) a1 += m; else a0 += m;
  }
  const double t0 = block_sum(a0, sh);
  __syncthreads();
  const double t1 = block_sum(a1, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = t0;
    partials[gridDim.x + blockIdx.x] = t1;
    __threadfence();
    last = atomicAdd(&ctl->blocks_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s0 = 0.0, s1 = 0.0;
  for (uint32_t b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    s0 += __ldcg(partials + b);
    s1 += __ldcg(partials + gridDim.x + b);
  }
  const double p0 = block_sum(s0, sh);
  __syncthreads();
  const double p1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    const double total = p0 + p1;
    const bool one = r * total < p1;
    const double pk = one ? p1 : p0;
    res[0] = one ? 1.0 : 0.0;
    res[1] = total > 0.0 ? pk / total : 0.0;
    res[2] = pk > 0.0 ? 1.0 / sqrt(pk) : 0.0;
    ctl->blocks_done = 0u;
  }
}

template <int KW>
__global__ void __launch_bounds__(256) k_collapse(Ctl* ctl, Bufs bufs, uint32_t word, uint64_t bit,
                                                  const double* res, uint32_t mg,
                                                  unsigned long long* plog) {
  __shared__ unsigned warp_cnt[32];
  __shared__ unsigned long long block_base;
  if (ctl->status != 0u) return;
  const uint64_t n = ctl->nnz;
  const unsigned cur = ctl->cur;
  const SoA s = pick(bufs, cur);
  const SoA out = pick(bufs, cur ^ 1u);
  if (blockIdx.x == 0 && threadIdx.x == 0) reset_label_masks(ctl, mg_rs(mg));
  const bool one = __ldcg(res) != 0.0;
  const double scale = __ldcg(res + 2);
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned nwarps = blockDim.x >> 5;
  uint64_t mo0 = 0, mo1 = 0, ma0 = ~0ull, ma1 = ~0ull;
  for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x; base < n;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    bool keep = false;
    uint64_t lo = 0, hi = 0;
    if (i < n) {
      lo = s.lo[i];
      hi = KW == 2 ? s.hi[i] : 0ull;
      keep = scale != 0.0 && ((((word ? hi : lo) & bit) != 0ull) == one);
    }
    const unsigned ballot = __ballot_sync(FULL, keep);
    if (lane == 0) warp_cnt[warp] = __popc(ballot);
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
      if (lane == 0) block_base = total ? atomicAdd(&ctl->out_count, (unsigned long long)total) : 0ull;
    }
    __syncthreads();
    if (keep) {
      const uint64_t pos = block_base + warp_cnt[warp] + __popc(ballot & ((1u << lane) - 1u));
      out.lo[pos] = lo;
      if (KW == 2) out.hi[pos] = hi;
      out.re[pos] = s.re[i] * scale;
      out.im[pos] = s.im[i] * scale;
      mo0 |= lo;
      mo1 |= hi;
      ma0 &= lo;
      ma1 &= hi;
    }
    __syncthreads();
  }
  merge_label_masks(ctl, mg_wr(mg), mo0, mo1, ma0, ma1);
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&ctl->blocks_done, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      const unsigned long long total = atomicAdd(&ctl->out_count, 0ull);
      ctl->nnz = total;        // never more than before: the buffers hold it
      ctl->cur = cur ^ 1u;
      ctl->updates += n;
      if (plog) {
        plog[0] = n;
        plog[1] = total;
      }
      ctl->out_count = 0ull;
      ctl->blocks_done = 0u;
      __threadfence();
    }
  }
}

__global__ void k_set_nnz(Ctl* ctl, unsigned long long nnz, uint32_t mg) {
  ctl->nnz = nnz;
  ctl->cur = 0u;
  ctl->status = 0u;
  ctl->out_count = 0ull;
  ctl->blocks_done = 0u;
  unknown_label_masks(ctl, mg_wr(mg));   // labels not inspected
  reset_label_masks(ctl, mg_rs(mg));
}

// |0...0>: one entry (label 0, amplitude 1) in buffer 0.
__global__ void k_reset_state(Ctl* ctl, Bufs bufs, int key_words, uint32_t mg) {
  bufs.b[0].lo[0] = 0ull;
  if (key_words == 2) bufs.b[0].hi[0] = 0ull;
  bufs.b[0].re[0] = 1.0;
  bufs.b[0].im[0] = 0.0;
  ctl->nnz = 1ull;
  ctl->cur = 0u;
  ctl->status = 0u;
  ctl->updates = 0ull;
  ctl->fail_pass = 0u;
  ctl->fail_gate = 0ull;
  ctl->out_count = 0ull;
  ctl->blocks_done = 0u;
  set_label_masks(ctl, mg_wr(mg), 0ull, 0ull, 0ull, 0ull);   // the single label 0
  reset_label_masks(ctl, mg_rs(mg));
}

// After a failed pass: passes that failed or were skipped left the mask
// buffers out of step with the state, so all three claim nothing.
__global__ void k_reset_status(Ctl* ctl) {
  ctl->status = 0u;
  ctl->fail_pass = 0u;
  ctl->fail_gate = 0ull;
  ctl->out_count = 0ull;
  ctl->blocks_done = 0u;
  ctl->grid_bar = 0u;   // a barrier that timed out left blocks counted
  for (uint32_t b = 0; b < 3; ++b) unknown_label_masks(ctl, b);
}

// Flags labels outside the register; unless mg is kNoMasks also merges the
// OR/AND masks of the uploaded labels.
template <int KW>
__global__ void k_check_labels(Ctl* ctl, Bufs bufs, uint64_t lim0, uint64_t lim1, unsigned* bad,
                               uint32_t mg) {
  const uint64_t n = ctl->nnz;
  if (mg != kNoMasks && blockIdx.x == 0 && threadIdx.x == 0) reset_label_masks(ctl, mg_rs(mg));
  const SoA s = pick(bufs, ctl->cur);
  uint64_t mo0 = 0, mo1 = 0, ma0 = ~0ull, ma1 = ~0ull;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k0 = s.lo[i];
    const uint64_t k1 = KW == 2 ? s.hi[i] : 0ull;
    if ((k0 & ~lim0) != 0ull || (k1 & ~lim1) != 0ull) atomicOr(bad, 1u);
    mo0 |= k0;
    mo1 |= k1;
    ma0 &= k0;
    ma1 &= k1;
  }
  if (mg != kNoMasks) merge_label_masks(ctl, mg_wr(mg), mo0, mo1, ma0, ma1);
}

// lc.max_blocks is the SM count times the resident blocks of lc.threads threads
int sm_count(const LaunchCfg& lc) {
  const int s = (int)((int64_t)lc.max_blocks * lc.threads / 2048);
  return s > 0 ? s : 1;
}

int grid_for(uint64_t work, int threads, int max_blocks) {
  uint64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (uint64_t)max_blocks) b = max_blocks;
  return (int)b;
}

// Shared memory of one block of the bit-sliced pass: 4 warps, each a tile of
// rows x (G + 1) words.
constexpr int kBsWarps = 4;
size_t bs_block_smem(uint32_t rows, uint32_t G) {
  return (size_t)kBsWarps * rows * (G + 1) * 4;
}
// Resident blocks per SM for a tile of G groups (registers and shared memory,
// as the runtime computes them).
template <int KW, int NW>
int bs_blocks_per_sm(uint32_t rows, uint32_t G) {
  const size_t smem = bs_block_smem(rows, G);
  if (smem > 200 * 1024) return 0;
  if (cudaFuncSetAttribute(k_fused_bs<KW, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int k = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, k_fused_bs<KW, NW>, kBsWarps * 32, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return k;
}

template <int KW, int NW>
int fused_bs_kw(const LaunchCfg& lc, Ctl* ctl, Bufs bufs, const BsLaunch& b, uint64_t nnz_bound,
                unsigned long long* plog) {
  const BsPass& P = *b.plan;
  if (P.op_words() > kBsMaxOps || P.nrows > 250) return 0;
  const int sms = sm_count(lc);
  // groups per tile: the most (fewest instructions per entry) that still give
  // every resident warp at least two tiles
  uint32_t G = b.groups;
  if (G == 0) {
    G = 4;
    for (uint32_t g = 32; g >= 8; g >>= 1) {
      const uint64_t tiles = (nnz_bound + 32ull * g - 1) / (32ull * g);
      const uint64_t resident = (uint64_t)sms * bs_blocks_per_sm<KW, NW>(P.nrows, g) * kBsWarps;
      if (tiles >= 2 * resident) {
        G = g;
        break;
      }
    }
  }
  if (G < 2) G = 2;
  if (G > 32) G = 32;
  const int bps = bs_blocks_per_sm<KW, NW>(P.nrows, G);
  if (bps < 1) return 0;
  static thread_local BsArgs a;   // 16 KB of ops: keep it off the stack
  std::memset(&a, 0, sizeof(a) - sizeof(a.ops));
  static_assert(sizeof(BsArgs) < 32000, "kernel parameters must stay under 32 KB");
  const uint32_t S = G + 1;
  const uint32_t rb = 4u * S;     // bytes per row of a tile column
  a.ngates = b.ngates;
  a.groups = G;
  a.stride = S;
  a.rows = P.nrows;
  a.word_out = P.word_out;
  for (uint32_t w = 0; w < 4; ++w) {
    a.word_bits[w] = P.word_bits[w];
    for (uint32_t j = 0; j < 32; ++j) a.row_of[w][j] = P.row_of[w][j];
  }
  a.aux_row0 = P.aux_row0;
  a.naux = P.aux_bits;
  a.ones_row = P.ones_row;
  a.has_perm = b.has_perm;
  a.has_phase = b.has_phase && P.aux_bits > 0;
  a.has_cnt = P.has_cnt ? 1u : 0u;
  a.nchunks = P.nchunks;
  uint64_t toff = 0;
  for (uint32_t c = 0; c < P.nchunks; ++c) {
    a.chunk_shift[c] = P.chunk_shift[c];
    a.chunk_bits[c] = P.chunk_bits[c];
    a.tables[c] = reinterpret_cast<const longlong2*>(b.tables) + toff;
    toff += 1ull << P.chunk_bits[c];
  }
  a.direct = P.direct ? reinterpret_cast<const double2*>(b.tables) + P.direct_offset() : nullptr;
  a.mg = b.mg;
  a.fallback = b.fallback;
  auto off = [&](uint8_t r) -> uint32_t { return r == kNoRow ? 0u : (uint32_t)r * rb; };
  uint32_t nw = 0;
  for (size_t j = 0; j < P.ops.size(); ++j) {
    const SOp& o = P.ops[j];
    const bool general = o.kind != SOP_FLIP;
    if (nw + (general && o.kind != SOP_AND ? 2u : 1u) > kBsMaxOps) return 0;
    uint4 w;
    w.x = off(o.c[0]);
    w.y = off(o.c[1]);
    w.z = off(o.c[2]);
    w.w = off(o.t) | (general ? (kBsGeneral | ((uint32_t)o.kind << 24)) : 0u);
    a.ops[nw++] = w;
    if (general && o.kind != SOP_AND) {
      uint4 e;
      e.x = off(o.s);
      e.y = off(o.f0);
      e.z = off(o.f1);
      e.w = (uint32_t)(o.a0 & 7u) | ((uint32_t)(o.a1 & 7u) << 8);
      a.ops[nw++] = e;
    }
  }
  a.nwords = nw;
  cudaStream_t st = (cudaStream_t)lc.stream;
  const int launched = b.build_tables ? launch_bs_tables(lc, b) : 0;
  if (launched < 0) return -1;
  const size_t smem = bs_block_smem(P.nrows, G);
  const uint64_t tiles = (nnz_bound + 32ull * G - 1) / (32ull * G);
  uint64_t blocks = (tiles + kBsWarps - 1) / kBsWarps;
  const uint64_t max_blocks = (uint64_t)sms * bps;
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  cudaFuncSetAttribute(k_fused_bs<KW, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_fused_bs<KW, NW><<<(int)blocks, kBsWarps * 32, smem, st>>>(ctl, bufs, a, plog);
  return cudaPeekAtLastError() == cudaSuccess ? launched + 1 : -1;
}

BranchArgs branch_args(const BranchLaunch& b) {
  BranchArgs a;
  a.op = b.op;
  a.eps2 = b.eps * b.eps;
  a.eps = b.eps;
  a.capacity = b.capacity;
  a.fail_tag = b.fail_tag;
  a.load_pct = b.load_pct;
  a.max_log2 = b.max_log2;
  a.probe_limit = b.probe_limit;
  a.pass_serial = b.pass_serial;
  a.mg = b.mg;
  return a;
}

}  // namespace

int launch_table_clear(const LaunchCfg& lc, Slot* table, uint64_t nslots) {
  const int blocks = grid_for(nslots, lc.threads, lc.max_blocks);
  k_table_clear<<<blocks, lc.threads, 0, (cudaStream_t)lc.stream>>>(table, nslots);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_fused(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, const Pass& p,
                 const OpWord* words, const double* ftab, uint64_t nnz_bound, uint32_t mg,
                 int lanes, uint32_t fallback, unsigned long long* plog) {
  if (p.ops.empty()) {   // every gate resolved on the host: only the update count
    k_count_updates<<<1, 1, 0, (cudaStream_t)lc.stream>>>(ctl, p.ngates, fallback);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
  }
  FusedArgs a;
  a.fallback = fallback;
  a.words = reinterpret_cast<const uint4*>(words);
  a.ftab = reinterpret_cast<const double2*>(ftab);
  a.nwords = (uint32_t)p.words.size();
  a.ngates = p.ngates;
  a.has_perm = p.has_perm;
  a.has_phase = p.has_phase;
  a.mg = mg;
  // labels per thread: as many as still leave about four warps per SM per
  // label slot (SPS_OPT_FUSED_LABELS overrides)
  int e = lanes;
  if (e == 0) {
    const uint64_t warps_wanted = 4ull * (uint64_t)sm_count(lc);
    e = 1;
    while (e < 8 && nnz_bound / (32ull * (uint64_t)(2 * e)) >= warps_wanted) e *= 2;
  }
  const int blocks = grid_for((nnz_bound + e - 1) / e, lc.threads, lc.max_blocks);
  // at most 4 words per op: <= 32 KB, under the default 48 KB
  const size_t smem = 16 * (size_t)a.nwords;
  cudaStream_t st = (cudaStream_t)lc.stream;
  if (key_words == 1) {
    if (e == 1) k_fused<1, 1><<<blocks, lc.threads, smem, st>>>(ctl, bufs, a, plog);
    else if (e == 2) k_fused<1, 2><<<blocks, lc.threads, smem, st>>>(ctl, bufs, a, plog);
    else if (e == 4) k_fused<1, 4><<<blocks, lc.threads, smem, st>>>(ctl, bufs, a, plog);
    else k_fused<1, 8><<<blocks, lc.threads, smem, st>>>(ctl, bufs, a, plog);
  } else {
    if (e == 1) k_fused<2, 1><<<blocks, lc.threads, smem, st>>>(ctl, bufs, a, plog);
    else if (e == 2) k_fused<2, 2><<<blocks, lc.threads, smem, st>>>(ctl, bufs, a, plog);
    else if (e == 4) k_fused<2, 4><<<blocks, lc.threads, smem, st>>>(ctl, bufs, a, plog);
    else k_fused<2, 8><<<blocks, lc.threads, smem, st>>>(ctl, bufs, a, plog);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_bs_tables(const LaunchCfg& lc, const BsLaunch& b) {
  const BsPass& P = *b.plan;
  if (!(b.has_phase && P.aux_bits > 0)) return 0;
  uint64_t toff = 0;
  int launched = 0;
  for (uint32_t c = 0; c < P.nchunks; ++c) {
    const uint32_t size = 1u << P.chunk_bits[c];
    const int blocks = (int)((size + 255) / 256);
    k_bs_tables<<<blocks, 256, 0, (cudaStream_t)lc.stream>>>(
        reinterpret_cast<const longlong2*>(b.factors), reinterpret_cast<longlong2*>(b.tables) + toff,
        P.chunk_bits[c], P.chunk_shift[c]);
    toff += size;
    ++launched;
  }
  if (P.direct) {
    const uint32_t size = 1u << P.aux_bits;
    const longlong2* t = reinterpret_cast<const longlong2*>(b.tables);
    k_bs_direct_table<<<(int)((size + 255) / 256), 256, 0, (cudaStream_t)lc.stream>>>(
        t, P.nchunks > 1 ? t + (1ull << P.chunk_bits[0]) : t, P.chunk_bits[0], P.aux_bits,
        reinterpret_cast<double2*>(b.tables) + P.direct_offset(), P.expand ? 1u : 0u, P.c_re,
        P.c_im);
    ++launched;
  }
  return cudaPeekAtLastError() == cudaSuccess ? launched : -1;
}

int launch_fused_bs(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, const BsLaunch& b,
                    uint64_t nnz_bound, unsigned long long* plog) {
  if (b.plan == nullptr || b.plan->ops.empty()) return 0;
  const uint32_t nw = b.plan->nw;
  if (key_words == 1)
    return nw <= 1 ? fused_bs_kw<1, 1>(lc, ctl, bufs, b, nnz_bound, plog)
                   : fused_bs_kw<1, 2>(lc, ctl, bufs, b, nnz_bound, plog);
  if (nw <= 2) return fused_bs_kw<2, 2>(lc, ctl, bufs, b, nnz_bound, plog);
  return nw == 3 ? fused_bs_kw<2, 3>(lc, ctl, bufs, b, nnz_bound, plog)
                 : fused_bs_kw<2, 4>(lc, ctl, bufs, b, nnz_bound, plog);
}

int launch_branch_emit(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, Slot* table,
                       const BranchLaunch& b, uint64_t nnz_bound, unsigned long long* plog) {
  const BranchArgs a = branch_args(b);
  cudaStream_t st = (cudaStream_t)lc.stream;
  const int blocks = grid_for(nnz_bound, lc.threads, lc.max_blocks);
  // lanes probing one insert together (SPS_OPT_COOP_WIDTH)
  auto go = [&](auto kern) { kern<<<blocks, lc.threads, 0, st>>>(ctl, bufs, table, a, plog); };
  if (key_words == 1) {
    if (b.coop == 8) go(k_branch_emit<1, 8>);
    else if (b.coop == 4) go(k_branch_emit<1, 4>);
    else if (b.coop == 2) go(k_branch_emit<1, 2>);
    else go(k_branch_emit<1, 1>);
  } else {
    if (b.coop == 8) go(k_branch_emit<2, 8>);
    else if (b.coop == 4) go(k_branch_emit<2, 4>);
    else if (b.coop == 2) go(k_branch_emit<2, 2>);
    else go(k_branch_emit<2, 1>);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_branch_compact(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, Slot* table,
                          const BranchLaunch& b, uint64_t nnz_bound, unsigned long long* plog) {
  const BranchArgs a = branch_args(b);
  cudaStream_t st = (cudaStream_t)lc.stream;
  const uint64_t tsize = 1ull << table_log2_for(nnz_bound, b.load_pct, b.max_log2);
  const int blocks = grid_for(tsize, lc.threads, lc.max_blocks);
  if (key_words == 1)
    k_branch_compact<1><<<blocks, lc.threads, 0, st>>>(ctl, bufs, table, a, plog);
  else
    k_branch_compact<2><<<blocks, lc.threads, 0, st>>>(ctl, bufs, table, a, plog);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_probability(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs,
                       uint64_t mask_lo, uint64_t mask_hi, uint64_t val_lo, uint64_t val_hi,
                       double* partials, int nblocks, double* result,
                       unsigned long long* plog) {
  cudaStream_t st = (cudaStream_t)lc.stream;
  const bool hi = key_words == 2 && (mask_hi | val_hi) != 0ull;
  if (key_words == 1)
    k_probability<1, false><<<nblocks, 256, 0, st>>>(ctl, bufs, mask_lo, mask_hi, val_lo, val_hi,
                                                     partials, result, plog);
  else if (hi)
    k_probability<2, true><<<nblocks, 256, 0, st>>>(ctl, bufs, mask_lo, mask_hi, val_lo, val_hi,
                                                    partials, result, plog);
  else
    k_probability<2, false><<<nblocks, 256, 0, st>>>(ctl, bufs, mask_lo, mask_hi, val_lo, val_hi,
                                                     partials, result, plog);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_measure(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, uint32_t qubit,
                   double r, double* partials, int nblocks, double* res, uint64_t nnz_bound,
                   uint32_t mg, unsigned long long* plog) {
  cudaStream_t st = (cudaStream_t)lc.stream;
  const uint32_t word = qubit >> 6;
  const uint64_t bit = 1ull << (qubit & 63u);
  const int blocks = grid_for(nnz_bound, lc.threads, lc.max_blocks);
  if (key_words == 1) {
    k_measure_sum<1><<<nblocks, 256, 0, st>>>(ctl, bufs, word, bit, r, partials, res);
    k_collapse<1><<<blocks, lc.threads, 0, st>>>(ctl, bufs, word, bit, res, mg, plog);
  } else {
    k_measure_sum<2><<<nblocks, 256, 0, st>>>(ctl, bufs, word, bit, r, partials, res);
    k_collapse<2><<<blocks, lc.threads, 0, st>>>(ctl, bufs, word, bit, res, mg, plog);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

int launch_set_nnz(void* stream, Ctl* ctl, unsigned long long nnz, uint32_t mg) {
  k_set_nnz<<<1, 1, 0, (cudaStream_t)stream>>>(ctl, nnz, mg);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_reset_state(void* stream, int key_words, Ctl* ctl, Bufs bufs, uint32_t mg) {
  k_reset_state<<<1, 1, 0, (cudaStream_t)stream>>>(ctl, bufs, key_words, mg);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_reset_status(void* stream, Ctl* ctl) {
  k_reset_status<<<1, 1, 0, (cudaStream_t)stream>>>(ctl);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_check_labels(void* stream, int key_words, Ctl* ctl, Bufs bufs, uint64_t lim_lo,
                        uint64_t lim_hi, unsigned int* bad_flag, uint64_t n, uint32_t mg) {
  const int blocks = grid_for(n, 256, 1024);
  if (key_words == 1)
    k_check_labels<1><<<blocks, 256, 0, (cudaStream_t)stream>>>(ctl, bufs, lim_lo, lim_hi, bad_flag,
                                                                 mg);
  else
    k_check_labels<2><<<blocks, 256, 0, (cudaStream_t)stream>>>(ctl, bufs, lim_lo, lim_hi, bad_flag,
                                                                 mg);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace sps
