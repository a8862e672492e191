// Bit-sliced fused pass (Sec. 3.2: a run of phase/permutation gates applied in
// one pass over the entries) compiled for one run at run time.
//
// The general bit-sliced kernel (sps_kernels.cu) reads each op from a list and
// walks it on shared-memory planes: every op costs a dependent chain of
// shared-memory loads and a store, plus decode and address arithmetic. Here the
// run is turned into CUDA source in which the walk is straight-line code on
// registers (a Toffoli is one three-input logic instruction on 32 entries) and
// every row offset, word count and table shape is a constant, compiled with
// NVRTC for the device's architecture and cached per source text. NVRTC is
// loaded at first use; without it, or if a compile fails, callers take the
// general kernel, which computes the same result.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "sps_internal.h"

namespace sps {
namespace {

// ---- NVRTC, resolved at first use ---------------------------------------------
struct Nvrtc {
  typedef int (*create_t)(void**, const char*, const char*, int, const char* const*,
                          const char* const*);
  typedef int (*compile_t)(void*, int, const char* const*);
  typedef int (*size_t_)(void*, size_t*);
  typedef int (*get_t)(void*, char*);
  typedef int (*destroy_t)(void**);
  create_t create = nullptr;
  compile_t compile = nullptr;
  size_t_ cubin_size = nullptr;
  get_t cubin = nullptr;
  size_t_ log_size = nullptr;
  get_t log = nullptr;
  destroy_t destroy = nullptr;
  bool ok = false;
};

Nvrtc* nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"};
    void* h = nullptr;
    for (const char* nm : names) {
      h = dlopen(nm, RTLD_NOW | RTLD_LOCAL);
      if (h) break;
    }
    if (!h) return;
    n.create = (Nvrtc::create_t)dlsym(h, "nvrtcCreateProgram");
    n.compile = (Nvrtc::compile_t)dlsym(h, "nvrtcCompileProgram");
    n.cubin_size = (Nvrtc::size_t_)dlsym(h, "nvrtcGetCUBINSize");
    n.cubin = (Nvrtc::get_t)dlsym(h, "nvrtcGetCUBIN");
    n.log_size = (Nvrtc::size_t_)dlsym(h, "nvrtcGetProgramLogSize");
    n.log = (Nvrtc::get_t)dlsym(h, "nvrtcGetProgramLog");
    n.destroy = (Nvrtc::destroy_t)dlsym(h, "nvrtcDestroyProgram");
    n.ok = n.create && n.compile && n.cubin_size && n.cubin && n.log_size && n.log && n.destroy;
  });
  return &n;
}

// Compiles `src` for sm_<major><minor>a; returns the cubin or an empty string
// (log receives the compiler's messages).
std::string compile_cubin(const std::string& src, int major, int minor, std::string* log) {
  Nvrtc* nv = nvrtc();
  if (!nv->ok) {
    if (log) *log = "runtime compiler not found";
    return std::string();
  }
  void* prog = nullptr;
  if (nv->create(&prog, src.c_str(), "sps_bs_jit.cu", 0, nullptr, nullptr) != 0) return std::string();
  char arch[64];
  std::snprintf(arch, sizeof(arch), "--gpu-architecture=sm_%d%da", major, minor);
  const char* opts[] = {arch, "-std=c++17", "--device-as-default-execution-space"};
  const int rc = nv->compile(prog, 3, opts);
  if (log) {
    size_t n = 0;
    nv->log_size(prog, &n);
    log->assign(n, '\0');
    if (n) nv->log(prog, &(*log)[0]);
  }
  std::string out;
  if (rc == 0) {
    size_t n = 0;
    nv->cubin_size(prog, &n);
    out.assign(n, '\0');
    if (n) nv->cubin(prog, &out[0]);
  }
  nv->destroy(&prog);
  return out;
}

// ---- the kernel template --------------------------------------------------------
// Constants and the walk are prepended by make_source(). Everything else is
// the general kernel's three phases with the constants folded in.
const char* kTemplate = R"JIT(
typedef unsigned int u32;
typedef unsigned long long u64;
typedef long long i64;
#define FULL 0xFFFFFFFFu

struct Soa { u64* lo; u64* hi; double* re; double* im; };
struct JArgs {
  unsigned char* ctl;
  Soa b[2];
  const longlong2* tab[4];
  const double2* direct;
  u64* plog;
  u32 fallback, mg_wr, mg_rs, ngates;
  // with RD: the readout's block sums and its total
  double* rd_part;
  double* rd_out;
};

struct Transposer {
  u32 rot[5], keep[5];
  __device__ __forceinline__ void init(unsigned lane) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const u32 m = 16u >> i;
      const u32 mk = i == 0 ? 0x0000FFFFu : i == 1 ? 0x00FF00FFu : i == 2 ? 0x0F0F0F0Fu
                   : i == 3 ? 0x33333333u : 0x55555555u;
      const bool upper = (lane & m) != 0u;
      rot[i] = upper ? 32u - m : m;
      keep[i] = upper ? ~mk : mk;
    }
  }
  __device__ __forceinline__ u32 operator()(u32 x) const {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const u32 y = __shfl_xor_sync(FULL, x, 16u >> i);
      const u32 t = __funnelshift_l(y, y, rot[i]);
      x = (x & keep[i]) | (t & ~keep[i]);
    }
    return x;
  }
};

__device__ __forceinline__ void cnt_add(u32& c0, u32& c1, u32& c2, u32 k, u32 f) {
  if (k & 1u) {
    const u32 carry0 = c0 & f;
    c0 ^= f;
    const u32 carry1 = c1 & carry0;
    c1 ^= carry0;
    c2 ^= carry1;
  }
  if (k & 2u) {
    const u32 carry1 = c1 & f;
    c1 ^= f;
    c2 ^= carry1;
  }
  if (k & 4u) c2 ^= f;
}

__device__ __forceinline__ void qmul(i64& ar, i64& ai, i64 br, i64 bi) {
  const i64 k1 = __mul64hi(br, ar + ai);
  const i64 k2 = __mul64hi(ar, bi - br);
  const i64 k3 = __mul64hi(ai, br + bi);
  ar = k1 - k3;
  ai = k1 + k2;
}

__device__ __forceinline__ double q_to_double(i64 v, int q) {
  if (v == 0) return 0.0;
  const u64 sgn = v < 0 ? 0x8000000000000000ull : 0ull;
  u64 m = v < 0 ? 0ull - (u64)v : (u64)v;
  const int lz = __clzll((i64)m);
  m <<= lz;
  u64 r = (m >> 11) + ((m >> 10) & 1ull);
  int e = 63 - lz - q;
  if (r >> 53) {
    r >>= 1;
    ++e;
  }
  return __longlong_as_double((i64)(sgn | ((u64)(e + 1023) << 52) | (r & 0x000FFFFFFFFFFFFFull)));
}

__device__ __forceinline__ u64* lm(unsigned char* ctl, u32 b, u32 stripe) {
  return reinterpret_cast<u64*>(ctl + OFF_LM) + ((u64)b * 32u + stripe) * 4u;
}

extern "C" __global__ void __launch_bounds__(128, LB_MIN) k_bs_jit(const JArgs a) {
  extern __shared__ __align__(16) u32 bsm[];
  __shared__ u64 part[4][32];
  unsigned char* ctl = a.ctl;
#if EXPAND && RD
  __shared__ double rsum[32];
  __shared__ u32 am_last;
  double racc = 0.0;   // this lane's readout sum
#endif
#if EXPAND
  // the expansion's 2^EX_D outputs from |0...0> (a reset not yet carried out):
  // nothing is read, the outputs go to buffer 1, the last block publishes them
  const u64 n = 1ull << EX_D;
  if (a.plog && blockIdx.x == 0 && threadIdx.x == 0) {
    a.plog[0] = 1ull;
    a.plog[1] = n;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
#else
  const u64 n = *reinterpret_cast<volatile u64*>(ctl + OFF_NNZ);
  const bool skip = a.fallback != 0u && *reinterpret_cast<volatile u32*>(ctl + OFF_AMP_STATE) == 1u;
  if (a.plog && blockIdx.x == 0 && threadIdx.x == 0) {
    a.plog[0] = skip ? 0ull : n;
    a.plog[1] = n;
  }
  if (*reinterpret_cast<volatile u32*>(ctl + OFF_STATUS) != 0u || skip) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *reinterpret_cast<u64*>(ctl + OFF_UPDATES) += n * a.ngates;
#endif
    if (HAS_PERM)
      for (u32 i = 0; i < 32u; ++i) {
        u64* p = lm(ctl, a.mg_rs, i);
        p[0] = 0ull;
        p[1] = 0ull;
        p[2] = ~0ull;
        p[3] = ~0ull;
      }
  }
#if EXPAND
  const Soa s = a.b[1];
#else
  const u32 cur = *reinterpret_cast<volatile u32*>(ctl + OFF_CUR);
  const Soa s = cur ? a.b[1] : a.b[0];
#endif
  const unsigned lane = threadIdx.x & 31u;
  const unsigned warp = threadIdx.x >> 5;
  u32* pl = bsm + warp * (ROWS * SS);
  const u64 tile_entries = 32ull * GG;
  const u64 ntiles = (n + tile_entries - 1) / tile_entries;
  const u64 nwarps = (u64)gridDim.x * (blockDim.x >> 5);
  Transposer tr;
  tr.init(lane);
  int my_row[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) my_row[w] = ROW_OF[w][lane];
  const int aux0 = lane < NAUX ? (int)((AUX0 + lane) * SS) : -1;
  const int aux1 = lane + 32u < NAUX ? (int)((AUX0 + 32u + lane) * SS) : -1;
  u64 mo0 = 0, mo1 = 0, ma0 = ~0ull, ma1 = ~0ull;
  for (u64 tile = (u64)blockIdx.x * (blockDim.x >> 5) + warp; tile < ntiles; tile += nwarps) {
    const u64 base = tile * tile_entries;
    const u64 tile_n = n - base < tile_entries ? n - base : tile_entries;
#if !EXPAND
    if (HAS_PHASE)
      for (u64 off = 16ull * lane; off < tile_n; off += 512ull) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(s.re + base + off));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(s.im + base + off));
      }
    // 1. load and transpose, 8 groups at a time
#pragma unroll 1
    for (u32 g0 = 0; g0 < GG; g0 += LOAD_BATCH) {
      u64 lo[LOAD_BATCH], hi[LOAD_BATCH];
#pragma unroll
      for (u32 k = 0; k < LOAD_BATCH; ++k) {
        const u64 e = base + 32ull * (g0 + k) + lane;
        const bool valid = e < n;
        lo[k] = valid ? __ldcs(s.lo + e) : 0ull;
        hi[k] = (KW == 2 && valid) ? __ldcs(s.hi + e) : 0ull;
      }
#pragma unroll
      for (u32 k = 0; k < LOAD_BATCH; ++k) {
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          if (WORD_BITS(w) == 0u) continue;
          const u64 src = w < 2 ? lo[k] : hi[k];
          const u32 t = tr((u32)(src >> (32 * (w & 1))));
          if (my_row[w] >= 0) pl[my_row[w] + g0 + k] = t;
        }
      }
    }
    {
      const u64 nb = base + nwarps * tile_entries;
      if (nb < n) {
        const u64 nn = n - nb < tile_entries ? n - nb : tile_entries;
        for (u64 off = 16ull * lane; off < nn; off += 512ull) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(s.lo + nb + off));
          if (KW == 2) asm volatile("prefetch.global.L2 [%0];" ::"l"(s.hi + nb + off));
        }
      }
    }
#else
    (void)tile_n;
#endif
    __syncwarp();
    // 2. the walk, lane g on group g (in an expansion: from the generated planes)
    if (lane < GG) walk(pl + lane, base + 32ull * lane);
    __syncwarp();
#if EXPAND && RD
    // the readout's matches among lane g's group: the tested output planes
    // (bit e: entry base + 32 g + e), as stored by the walk
    u32 rmatch = 0u;
    if (!RD_NONE && lane < GG) {
      const u64 g0e = base + 32ull * lane;
      rmatch = FULL_TILES ? FULL
             : g0e >= n ? 0u : n - g0e >= 32ull ? FULL : (1u << (u32)(n - g0e)) - 1u;
      rmatch &= rd_match(pl + lane);
    }
#endif
    // 3. transpose back and store, 4 groups at a time
#pragma unroll 1
    for (u32 g0 = 0; g0 < GG; g0 += STORE_BATCH) {
      u64 aux[STORE_BATCH];
      u64 ent[STORE_BATCH];
#pragma unroll
      for (u32 k = 0; k < STORE_BATCH; ++k) {
        const u32 g = g0 + k;
        aux[k] = 0ull;
        ent[k] = base + 32ull * g + lane;
        const bool valid = FULL_TILES || ent[k] < n;
        if (HAS_PERM) {
          u64 lo = 0ull, hi = 0ull;
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            if (!((WORD_OUT >> w) & 1u)) continue;
            const u64 x = ((SPARSE_W >> w) & 1u)
                              ? (u64)sparse_word(w, pl, g, lane)
                              : (u64)tr(my_row[w] >= 0 ? pl[my_row[w] + g] : 0u);
            if (w < 2) lo |= x << (32 * w);
            else hi |= x << (32 * (w - 2));
          }
          if (valid) {
            if (EXPAND || (WORD_OUT & 3u)) s.lo[ent[k]] = lo;
            else lo = s.lo[ent[k]];
            if (KW == 2) {
              if (EXPAND || (WORD_OUT & 12u)) s.hi[ent[k]] = hi;
              else hi = s.hi[ent[k]];
            }
            mo0 |= lo;
            mo1 |= hi;
            ma0 &= lo;
            ma1 &= hi;
          }
        }
#if EXPAND
        if (!HAS_PHASE && valid) {   // no phase anywhere: the common factor
          s.re[ent[k]] = C_RE;
          s.im[ent[k]] = C_IM;
        }
#endif
        if (HAS_PHASE) {
          const u32 x0 = tr(aux0 >= 0 ? pl[aux0 + g] : 0u);
          const u32 x1 = NAUX > 32u ? tr(aux1 >= 0 ? pl[aux1 + g] : 0u) : 0u;
          aux[k] = valid ? ((u64)x0 | ((u64)x1 << 32)) : 0ull;
        }
      }
      if (HAS_PHASE && DIRECT) {   // one table of every aux pattern's phase
        double2 ph[STORE_BATCH];
        double re[STORE_BATCH], im[STORE_BATCH];
#pragma unroll
        for (u32 k = 0; k < STORE_BATCH; ++k) {
          ph[k] = make_double2(1.0, 0.0);
#if EXPAND
          // every output from the table (entry 0: the common factor itself)
          re[k] = C_RE;
          im[k] = C_IM;
          if (!FULL_TILES && ent[k] >= n) continue;
#else
          re[k] = im[k] = 0.0;
          if (aux[k] == 0ull) continue;
          re[k] = __ldcs(s.re + ent[k]);
          im[k] = __ldcs(s.im + ent[k]);
#endif
          ph[k] = __ldg(a.direct + aux[k]);
        }
#if EXPAND
        // the expansion's table holds the common factor times each phase
#pragma unroll
        for (u32 k = 0; k < STORE_BATCH; ++k) {
          if (!FULL_TILES && ent[k] >= n) continue;
          s.re[ent[k]] = ph[k].x;
          s.im[ent[k]] = ph[k].y;
        }
#else
        bool real = true;
#pragma unroll
        for (u32 k = 0; k < STORE_BATCH; ++k) real = real && (__double_as_longlong(im[k]) << 1) == 0;
        real = __all_sync(FULL, real);   // per warp: no predicated complex form
#pragma unroll
        for (u32 k = 0; k < STORE_BATCH; ++k) {
          if (aux[k] == 0ull) continue;
          if (real) {
            s.re[ent[k]] = re[k] * ph[k].x;
            s.im[ent[k]] = re[k] * ph[k].y;
          } else {
            s.re[ent[k]] = fma(re[k], ph[k].x, -(im[k] * ph[k].y));
            s.im[ent[k]] = fma(re[k], ph[k].y, im[k] * ph[k].x);
          }
        }
#endif
      } else if (HAS_PHASE) {
        double re[STORE_BATCH], im[STORE_BATCH];
        longlong2 t0[STORE_BATCH], t1[STORE_BATCH];
#pragma unroll
        for (u32 k = 0; k < STORE_BATCH; ++k) {
          re[k] = im[k] = 0.0;
          t0[k] = t1[k] = make_longlong2(0, 0);
          if (aux[k] == 0ull) continue;
          re[k] = __ldcs(s.re + ent[k]);
          im[k] = __ldcs(s.im + ent[k]);
          const u32 i0 = (u32)(aux[k] >> CSH0) & ((1u << CBITS0) - 1u);
          if (i0) t0[k] = __ldg(a.tab[0] + i0);
          if (NCHUNK > 1) {
            const u32 i1 = (u32)(aux[k] >> CSH1) & ((1u << CBITS1) - 1u);
            if (i1) t1[k] = __ldg(a.tab[1] + i1);
          }
        }
#pragma unroll
        for (u32 k = 0; k < STORE_BATCH; ++k) {
          if (aux[k] == 0ull) continue;
          i64 pr = 0, pi = 0;
          int q = 62;
          bool any = false;
          if ((u32)(aux[k] >> CSH0) & ((1u << CBITS0) - 1u)) {
            pr = t0[k].x;
            pi = t0[k].y;
            any = true;
          }
          if (NCHUNK > 1 && ((u32)(aux[k] >> CSH1) & ((1u << CBITS1) - 1u))) {
            if (any) {
              qmul(pr, pi, t1[k].x, t1[k].y);
              q -= 2;
            } else {
              pr = t1[k].x;
              pi = t1[k].y;
              any = true;
            }
          }
#pragma unroll
          for (int c = 2; c < NCHUNK; ++c) {
            const u32 idx = (u32)(aux[k] >> CSH(c)) & ((1u << CBITS(c)) - 1u);
            if (idx == 0u) continue;
            const longlong2 t = __ldg(a.tab[c] + idx);
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
#if EXPAND && RD
    // the matching entries' amplitudes, each read back by the lane that stored
    // it, over the groups with a match only, in group order (rare: FP64
    // products only in warps with a match)
    for (u32 gm = __ballot_sync(FULL, rmatch != 0u); gm != 0u; gm &= gm - 1u) {
      const u32 g = (u32)__ffs((int)gm) - 1u;
      const u32 mw = __shfl_sync(FULL, rmatch, g);
      if ((mw >> lane) & 1u) {
        const u64 e = base + 32ull * g + lane;
        const double re = s.re[e], im = s.im[e];
        racc += re * re + im * im;
      }
    }
#endif
    __syncwarp();
  }
  if (HAS_PERM) {
    // OR / AND of the written labels: block reduction, one stripe per block
    for (int d = 16; d > 0; d >>= 1) {
      mo0 |= __shfl_xor_sync(FULL, mo0, d);
      mo1 |= __shfl_xor_sync(FULL, mo1, d);
      ma0 &= __shfl_xor_sync(FULL, ma0, d);
      ma1 &= __shfl_xor_sync(FULL, ma1, d);
    }
    if (lane == 0) {
      part[0][warp] = mo0;
      part[1][warp] = mo1;
      part[2][warp] = ma0;
      part[3][warp] = ma1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (unsigned w = 1; w < (blockDim.x >> 5); ++w) {
        mo0 |= part[0][w];
        mo1 |= part[1][w];
        ma0 &= part[2][w];
        ma1 &= part[3][w];
      }
      u64* p = lm(ctl, a.mg_wr, blockIdx.x % 32u);
      if (mo0) atomicOr(p, mo0);
      if (mo1) atomicOr(p + 1, mo1);
      if (~ma0) atomicAnd(p + 2, ma0);
      if (~ma1) atomicAnd(p + 3, ma1);
    }
  }
#if EXPAND
  // the last block publishes the outputs and does the reset's work on the
  // control block (no status, no failure record; the updates of the expansion,
  // 2^EX_D - 1, and of the run, 2^EX_D per gate)
  // (with RD, first the readout: block sums in a fixed order, which the last
  // block adds in block order)
#if RD
  for (int d = 16; d > 0; d >>= 1) racc += __shfl_down_sync(FULL, racc, d);
  if (lane == 0) rsum[warp] = racc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (unsigned w = 0; w < (blockDim.x >> 5); ++w) t += rsum[w];
    a.rd_part[blockIdx.x] = t;
    __threadfence();
    const u32 done = atomicAdd(reinterpret_cast<u32*>(ctl + OFF_BLOCKS_DONE), 1u);
    am_last = done == gridDim.x - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
    double t = 0.0;
    for (u32 b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += __ldcg(a.rd_part + b);
    for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(FULL, t, d);
    __syncthreads();
    if (lane == 0) rsum[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = 0.0;
      for (unsigned w = 0; w < (blockDim.x >> 5); ++w) r += rsum[w];
      *a.rd_out = r;
    }
  }
  if (threadIdx.x == 0 && am_last) {
    {
#else
  if (threadIdx.x == 0) {
    __threadfence();
    const u32 done = atomicAdd(reinterpret_cast<u32*>(ctl + OFF_BLOCKS_DONE), 1u);
    if (done == gridDim.x - 1) {
#endif
      __threadfence();
      *reinterpret_cast<volatile u32*>(ctl + OFF_STATUS) = 0u;
      *reinterpret_cast<volatile u32*>(ctl + OFF_FAIL_PASS) = 0u;
      *reinterpret_cast<volatile u64*>(ctl + OFF_FAIL_GATE) = 0ull;
      *reinterpret_cast<volatile u64*>(ctl + OFF_UPDATES) = (n - 1ull) + n * a.ngates;
      *reinterpret_cast<volatile u64*>(ctl + OFF_NNZ) = n;
      *reinterpret_cast<volatile u32*>(ctl + OFF_CUR) = 1u;
      *reinterpret_cast<volatile u64*>(ctl + OFF_OUT_COUNT) = 0ull;
      *reinterpret_cast<volatile u32*>(ctl + OFF_BLOCKS_DONE) = 0u;
      __threadfence();
    }
  }
#endif
}
)JIT";

constexpr int kJitWarps = 4;

// A readout compiled into the expansion form: the output planes it tests
// (row offsets in words) and the wanted value of each; none: no output label
// can match. key(): its bytes, for the caches.
struct RdForm {
  bool none = false;
  std::vector<uint16_t> row;
  std::vector<uint8_t> want;
  std::string key() const {
    std::string k(1, none ? '\1' : '\0');
    k.append(reinterpret_cast<const char*>(row.data()), row.size() * sizeof(uint16_t));
    k.append(reinterpret_cast<const char*>(want.data()), want.size());
    return k;
  }
};

// The readout (mask, value) on the outputs of expansion plan P in tiles of G
// groups: a tested bit with a row is a plane; one without is 0 in every output
// label (the launch writes every word, and a bit without a row stays 0).
RdForm readout_form(const BsPass& P, int kw, uint32_t G, const uint64_t mask[2],
                    const uint64_t value[2]) {
  RdForm f;
  for (int i = 0; i < 128; ++i) {
    const uint64_t bit = 1ull << (i & 63);
    const bool m = (mask[i >> 6] & bit) != 0ull, v = (value[i >> 6] & bit) != 0ull;
    if (!m || i >= 64 * kw) {
      f.none = f.none || v;   // a wanted bit outside the mask or the label
      continue;
    }
    const int w = i >> 5;
    const uint8_t r = ((P.word_out >> w) & 1u) ? P.row_of[w][i & 31] : kNoRow;
    if (r == kNoRow) {
      f.none = f.none || v;
      continue;
    }
    f.row.push_back((uint16_t)(r * (G + 1)));
    f.want.push_back(v ? 1u : 0u);
  }
  return f;
}

// The constants and the walk of one plan for tiles of G groups (16 or 32),
// then the template. Tiles of 16 groups leave half the lanes idle in the walk
// and load and store in smaller batches.
std::string make_source(const BsPass& P, int kw, bool has_perm, bool has_phase, uint32_t G,
                        const RdForm* rd) {
  const uint32_t S = G + 1;
  std::string o;
  char buf[256];
  auto def = [&](const char* name, unsigned long long v) {
    std::snprintf(buf, sizeof(buf), "#define %s %lluu\n", name, v);
    o += buf;
  };
  def("KW", (unsigned)kw);
  def("NW", P.nw);
  def("GG", G);
  def("LB_MIN", 4);
  def("LOAD_BATCH", G >= 32 ? 8 : 4);
  def("STORE_BATCH", G >= 32 ? 4 : 2);
  def("SS", S);
  def("ROWS", P.nrows);
  def("AUX0", P.aux_row0);
  def("NAUX", P.aux_bits);
  def("HAS_PERM", (has_perm || P.expand) ? 1 : 0);
  def("EXPAND", P.expand ? 1 : 0);
  def("EX_D", P.ex_d);
  def("RD", rd && P.expand ? 1 : 0);
  // an expansion whose 2^EX_D outputs fill every tile: no entry test
  def("FULL_TILES", P.expand && P.ex_d < 64 && ((1ull << P.ex_d) % (32ull * G)) == 0 ? 1 : 0);
  def("RD_NONE", rd && rd->none ? 1 : 0);
  def("OFF_FAIL_PASS", offsetof(Ctl, fail_pass));
  def("OFF_FAIL_GATE", offsetof(Ctl, fail_gate));
  def("OFF_BLOCKS_DONE", offsetof(Ctl, blocks_done));
  def("OFF_OUT_COUNT", offsetof(Ctl, out_count));
  std::snprintf(buf, sizeof(buf), "#define C_RE %.17g\n#define C_IM %.17g\n", P.c_re, P.c_im);
  o += buf;
  def("HAS_PHASE", (has_phase && P.aux_bits > 0) ? 1 : 0);
  def("WORD_OUT", P.word_out);
  def("NCHUNK", P.nchunks);
  def("DIRECT", P.direct ? 1 : 0);
  def("OFF_NNZ", offsetof(Ctl, nnz));
  def("OFF_CUR", offsetof(Ctl, cur));
  def("OFF_STATUS", offsetof(Ctl, status));
  def("OFF_UPDATES", offsetof(Ctl, updates));
  def("OFF_AMP_STATE", offsetof(Ctl, amp_state));
  def("OFF_LM", offsetof(Ctl, lm));
  static_assert(sizeof(((Ctl*)nullptr)->lm[0][0]) == 32, "mask stripe layout");
  for (int c = 0; c < 4; ++c) {
    std::snprintf(buf, sizeof(buf), "#define CSH%d %uu\n#define CBITS%d %uu\n", c,
                  c < (int)P.nchunks ? P.chunk_shift[c] : 0u, c,
                  c < (int)P.nchunks ? P.chunk_bits[c] : 1u);
    o += buf;
  }
  o += "#define CSH(c) ((c) == 0 ? CSH0 : (c) == 1 ? CSH1 : (c) == 2 ? CSH2 : CSH3)\n";
  o += "#define CBITS(c) ((c) == 0 ? CBITS0 : (c) == 1 ? CBITS1 : (c) == 2 ? CBITS2 : CBITS3)\n";
  std::snprintf(buf, sizeof(buf),
                "#define WORD_BITS(w) ((w) == 0 ? %uu : (w) == 1 ? %uu : (w) == 2 ? %uu : %uu)\n",
                P.word_bits[0], P.word_bits[1], P.word_bits[2], P.word_bits[3]);
  o += buf;
  // row offsets (in words) of each lane's bit, -1 without a row
  o += "__device__ const int ROW_OF[4][32] = {";
  for (int w = 0; w < 4; ++w) {
    o += w ? ",{" : "{";
    for (int j = 0; j < 32; ++j) {
      const uint8_t r = P.row_of[w][j];
      std::snprintf(buf, sizeof(buf), "%s%d", j ? "," : "", r == kNoRow ? -1 : (int)(r * S));
      o += buf;
    }
    o += "}";
  }
  o += "};\n";
  // forward declarations; the walk follows the template
  o += "__device__ __forceinline__ void walk(unsigned int* col, unsigned long long tb);\n";
  // the readout's test of 32 outputs: the AND of the tested planes, each
  // taken as is (wanted 1) or inverted (wanted 0)
  o += "__device__ __forceinline__ unsigned int rd_match(const unsigned int* col) {\n";
  o += "  unsigned int m = 0xFFFFFFFFu;\n";
  if (rd)
    for (size_t i = 0; i < rd->row.size(); ++i) {
      std::snprintf(buf, sizeof(buf), "  m &= %scol[%u];\n", rd->want[i] ? "" : "~",
                    (unsigned)rd->row[i]);
      o += buf;
    }
  o += "  return m;\n}\n";
  // words with at most 4 rows: each output bit read from its plane (one
  // broadcast load per row) instead of a 32 x 32 transpose
  uint32_t sparse = 0;
  for (uint32_t w = 0; w < 4; ++w)
    if (__builtin_popcount(P.word_bits[w]) <= 4) sparse |= 1u << w;
  def("SPARSE_W", sparse);
  o += "__device__ __forceinline__ unsigned int sparse_word(int w, const unsigned int* pl, "
       "unsigned int g, unsigned int lane) {\n  unsigned int x = 0u;\n";
  for (uint32_t w = 0; w < 4; ++w) {
    if (!((sparse >> w) & 1u) || P.word_bits[w] == 0u) continue;
    std::snprintf(buf, sizeof(buf), "  if (w == %u) {\n", w);
    o += buf;
    for (uint32_t j = 0; j < 32; ++j) {
      const uint8_t r = P.row_of[w][j];
      if (!((P.word_bits[w] >> j) & 1u) || r == kNoRow) continue;
      std::snprintf(buf, sizeof(buf), "    x |= ((pl[%u + g] >> lane) & 1u) << %u;\n",
                    (unsigned)(r * S), j);
      o += buf;
    }
    o += "  }\n";
  }
  o += "  return x;\n}\n";
  o += kTemplate;
  // ---- the walk: straight-line code on registers
  std::vector<uint8_t> read(256, 0), written(256, 0);
  const uint8_t ones = (uint8_t)P.ones_row;
  const uint8_t scratch = (uint8_t)(P.ones_row - 1u);
  for (const SOp& op : P.ops) {
    for (int k = 0; k < 3; ++k)
      if (op.c[k] != ones) read[op.c[k]] = 1;
    if (op.kind & SOP_SEL) read[op.s] = 1;
    if (op.kind & (SOP_FLIP | SOP_AND)) written[op.t] = 1;
    if (op.kind & SOP_FLIP) read[op.t] = 1;
  }
  o += "__device__ __forceinline__ void walk(unsigned int* col, unsigned long long tb) {\n";
  o += "  u32 c0 = 0u, c1 = 0u, c2 = 0u;\n";
  o += "  (void)tb;\n";
  // in an expansion every label row is generated: bit i of row r is choice bit
  // j of output tb + i (for j < 5 a fixed pattern, above it one bit of tb)
  static const char* kPat[5] = {"0xAAAAAAAAu", "0xCCCCCCCCu", "0xF0F0F0F0u", "0xFF00FF00u",
                                "0xFFFF0000u"};
  for (uint32_t r = 0; r < P.label_rows; ++r) {
    if (P.expand) {
      const int j = P.row_choice[r];
      if (j < 0)
        std::snprintf(buf, sizeof(buf), "  u32 p%u = 0u;\n", r);
      else if (j < 5)
        std::snprintf(buf, sizeof(buf), "  u32 p%u = %s;\n", r, kPat[j]);
      else
        std::snprintf(buf, sizeof(buf), "  u32 p%u = ((tb >> %d) & 1ull) ? 0xFFFFFFFFu : 0u;\n", r, j);
      o += buf;
      written[r] = 1;   // every label row is stored for the transposes back
    } else if (read[r] || written[r]) {
      std::snprintf(buf, sizeof(buf), "  u32 p%u = col[%u];\n", r, r * S);
      o += buf;
    }
  }
  std::snprintf(buf, sizeof(buf), "  u32 p%u = 0u;\n", (unsigned)scratch);
  o += buf;
  const uint32_t fire0 = P.aux_row0 + (P.has_cnt ? 3u : 0u);
  for (uint32_t r = fire0; r < P.aux_row0 + P.aux_bits; ++r) {
    std::snprintf(buf, sizeof(buf), "  u32 p%u = 0u;\n", r);
    o += buf;
  }
  auto cond = [&](const SOp& op) {
    std::string c;
    for (int k = 0; k < 3; ++k) {
      if (op.c[k] == ones) continue;
      std::snprintf(buf, sizeof(buf), "%sp%u", c.empty() ? "" : " & ", (unsigned)op.c[k]);
      c += buf;
    }
    return c.empty() ? std::string("0xFFFFFFFFu") : c;
  };
  for (const SOp& op : P.ops) {
    if (op.kind == SOP_FLIP) {
      o += "  p" + std::to_string(op.t) + " ^= " + cond(op) + ";\n";
      continue;
    }
    if (op.kind == SOP_AND) {
      o += "  p" + std::to_string(op.t) + " = " + cond(op) + ";\n";
      continue;
    }
    o += "  { const u32 f = " + cond(op) + ";\n";
    o += std::string("    const u32 sel = ") +
         ((op.kind & SOP_SEL) ? "p" + std::to_string(op.s) : std::string("0u")) + ";\n";
    if (op.kind & SOP_CNT) {
      o += "    cnt_add(c0, c1, c2, " + std::to_string(op.a0 & 7u) + "u, f & ~sel);\n";
      if (op.kind & SOP_SEL)
        o += "    cnt_add(c0, c1, c2, " + std::to_string(op.a1 & 7u) + "u, f & sel);\n";
    }
    if (op.kind & SOP_FIRE) {
      o += "    p" + std::to_string(op.f0) + " = f & ~sel;\n";
      if (op.kind & SOP_SEL) o += "    p" + std::to_string(op.f1) + " = f & sel;\n";
    }
    if (op.kind & SOP_FLIP) o += "    p" + std::to_string(op.t) + " ^= f;\n";
    o += "  }\n";
  }
  for (uint32_t r = 0; r < P.label_rows; ++r)
    if (written[r]) {
      std::snprintf(buf, sizeof(buf), "  col[%u] = p%u;\n", r * S, r);
      o += buf;
    }
  if (P.has_cnt) {
    std::snprintf(buf, sizeof(buf), "  col[%u] = c0;\n  col[%u] = c1;\n  col[%u] = c2;\n",
                  P.aux_row0 * S, (P.aux_row0 + 1) * S, (P.aux_row0 + 2) * S);
    o += buf;
  }
  for (uint32_t r = fire0; r < P.aux_row0 + P.aux_bits; ++r) {
    std::snprintf(buf, sizeof(buf), "  col[%u] = p%u;\n", r * S, r);
    o += buf;
  }
  o += "}\n";
  return o;
}

struct JitEntry {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kernel = nullptr;
  bool ok = false;
};

std::mutex g_jit_mu;
std::unordered_map<std::string, JitEntry>* g_jit = nullptr;

// The compiled kernel for `src` on the current device's architecture
// (compiled once per source text and architecture; a failure is remembered).
const JitEntry* jit_kernel(const std::string& src) {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const std::string key = std::to_string(major) + "." + std::to_string(minor) + "\n" + src;
  std::lock_guard<std::mutex> lk(g_jit_mu);
  if (!g_jit) g_jit = new std::unordered_map<std::string, JitEntry>();
  auto it = g_jit->find(key);
  if (it != g_jit->end()) return it->second.ok ? &it->second : nullptr;
  JitEntry e;
  std::string log;
  const std::string cubin = compile_cubin(src, major, minor, &log);
  if (!cubin.empty() &&
      cudaLibraryLoadData(&e.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) ==
          cudaSuccess &&
      cudaLibraryGetKernel(&e.kernel, e.lib, "k_bs_jit") == cudaSuccess)
    e.ok = true;
  cudaGetLastError();
  auto ins = g_jit->emplace(key, e).first;
  return ins->second.ok ? &ins->second : nullptr;
}

// The fields of a pass that decide its kernel's source (everything make_source
// reads: all but the phase factors, which reach the kernel as device tables),
// with the launch form and the architecture: the key of a second cache level
// that costs a copy of the fields instead of a source generation.
static_assert(sizeof(SOp) == 10, "SOp is ten bytes of rows and steps");
std::string content_key(const BsPass& P, int kw, bool has_perm, bool has_phase, uint32_t G,
                        int major, int minor) {
  std::string k;
  k.reserve(256 + P.ops.size() * sizeof(SOp) + P.row_choice.size());
  auto put = [&](const void* p, size_t n) { k.append(static_cast<const char*>(p), n); };
  const int32_t hdr[6] = {major, minor, kw, has_perm ? 1 : 0, has_phase ? 1 : 0, (int32_t)G};
  put(hdr, sizeof(hdr));
  const uint32_t f[8] = {P.nw, P.nrows, P.label_rows, P.aux_row0, P.aux_bits, P.ones_row,
                         P.word_out, P.nchunks};
  put(f, sizeof(f));
  const uint8_t flags[3] = {(uint8_t)P.has_cnt, (uint8_t)P.expand, (uint8_t)P.direct};
  put(flags, sizeof(flags));
  put(P.word_bits, sizeof(P.word_bits));
  put(P.row_of, sizeof(P.row_of));
  put(P.chunk_shift, sizeof(P.chunk_shift));
  put(P.chunk_bits, sizeof(P.chunk_bits));
  put(&P.c_re, sizeof(double));
  put(&P.c_im, sizeof(double));
  put(&P.ex_d, sizeof(P.ex_d));
  const uint32_t counts[2] = {(uint32_t)P.ops.size(), (uint32_t)P.row_choice.size()};
  put(counts, sizeof(counts));
  if (!P.ops.empty()) put(P.ops.data(), P.ops.size() * sizeof(SOp));
  if (!P.row_choice.empty()) put(P.row_choice.data(), P.row_choice.size());
  return k;
}

std::unordered_map<std::string, const JitEntry*>* g_jit_content = nullptr;

// The compiled kernel of a pass: from the cache of pass contents, else its
// source is generated and compiled (or found in the cache of sources).
const JitEntry* jit_kernel_for(const BsPass& P, int kw, bool has_perm, bool has_phase, uint32_t G,
                               const RdForm* rd) {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::string key = content_key(P, kw, has_perm, has_phase, G, major, minor);
  if (rd) key += "rd" + rd->key();
  {
    std::lock_guard<std::mutex> lk(g_jit_mu);
    if (!g_jit_content) g_jit_content = new std::unordered_map<std::string, const JitEntry*>();
    auto it = g_jit_content->find(key);
    if (it != g_jit_content->end()) return it->second;
  }
  const JitEntry* e = jit_kernel(make_source(P, kw, has_perm, has_phase, G, rd));
  std::lock_guard<std::mutex> lk(g_jit_mu);
  g_jit_content->emplace(key, e);
  return e;
}

}  // namespace

int launch_fused_bs_jit(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, const BsLaunch& b,
                        uint64_t nnz_bound, unsigned long long* plog) {
  const BsPass& P = *b.plan;
  if (P.ops.empty() || P.nrows > 250 || P.nchunks > 4) return 0;
  const int sms = lc.max_blocks * lc.threads / 2048 > 0 ? lc.max_blocks * lc.threads / 2048 : 1;
  // tiles of 32 groups: every lane walks; with 16 the register budget of the
  // extra resident blocks made the walk spill (SPS_OPT_BITSLICE_GROUPS 2..16
  // still asks for 16)
  const uint32_t G = (b.groups == 0 || b.groups >= 32) ? 32u : 16u;
  const size_t smem = (size_t)kJitWarps * P.nrows * (G + 1) * 4;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  // the form: device, label words, permutes, phases, tile groups
  const uint32_t form = 1u | ((uint32_t)dev << 8) | ((uint32_t)key_words << 16) |
                        (b.has_perm ? 1u << 20 : 0u) | (b.has_phase ? 1u << 21 : 0u) | (G << 24);
  // a readout is compiled into the expansion form (a kernel of its own)
  RdForm rdf;
  bool rd = b.rd && P.expand;
  std::string rkey;
  if (rd) {
    rdf = readout_form(P, key_words, G, b.rd->mask, b.rd->value);
    if (!rdf.none && rdf.row.size() < b.rd->min_planes) rd = false;   // a broad condition
    rkey = rdf.key();
  }
  const void* fn = nullptr;
  int bps = 0;
  if (!rd && P.jit_form == form) {
    fn = P.jit_fn;
    bps = P.jit_bps;
  } else if (rd && P.jit_rd_form == form && P.jit_rd_key == rkey) {
    fn = P.jit_rd_fn;
    bps = P.jit_rd_bps;
  }
  if (!fn) {
    const JitEntry* e =
        jit_kernel_for(P, key_words, b.has_perm != 0, b.has_phase != 0, G, rd ? &rdf : nullptr);
    if (!e) return 0;
    fn = reinterpret_cast<const void*>(e->kernel);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kJitWarps * 32, smem) !=
            cudaSuccess ||
        bps < 1) {
      cudaGetLastError();
      return 0;
    }
    if (rd) {
      P.jit_rd_form = form;
      P.jit_rd_key = rkey;
      P.jit_rd_fn = fn;
      P.jit_rd_bps = bps;
    } else {
      P.jit_form = form;
      P.jit_fn = fn;
      P.jit_bps = bps;
    }
  }
  const int launched = b.build_tables ? launch_bs_tables(lc, b) : 0;
  if (launched < 0) return -1;
  struct Soa { uint64_t* lo; uint64_t* hi; double* re; double* im; };
  struct JArgs {
    unsigned char* ctl;
    Soa b[2];
    const void* tab[4];
    const void* direct;
    unsigned long long* plog;
    uint32_t fallback, mg_wr, mg_rs, ngates;
    double* rd_part;
    double* rd_out;
  } args;
  std::memset(&args, 0, sizeof(args));
  args.ctl = reinterpret_cast<unsigned char*>(ctl);
  for (int k = 0; k < 2; ++k) args.b[k] = Soa{bufs.b[k].lo, bufs.b[k].hi, bufs.b[k].re, bufs.b[k].im};
  uint64_t toff = 0;
  for (uint32_t c = 0; c < P.nchunks; ++c) {
    args.tab[c] = reinterpret_cast<const char*>(b.tables) + 16 * toff;
    toff += 1ull << P.chunk_bits[c];
  }
  args.direct = P.direct ? reinterpret_cast<const char*>(b.tables) + 16 * P.direct_offset() : nullptr;
  args.plog = plog;
  args.fallback = b.fallback;
  args.mg_wr = mg_wr(b.mg);
  args.mg_rs = mg_rs(b.mg);
  args.ngates = b.ngates;
  const uint64_t tiles = (nnz_bound + 32ull * G - 1) / (32ull * G);
  uint64_t blocks = (tiles + kJitWarps - 1) / kJitWarps;
  const uint64_t max_blocks = (uint64_t)sms * bps;
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  if (rd) {   // one block sum each: at most cap blocks (the tiles are grid-strided)
    if (blocks > b.rd->cap) blocks = b.rd->cap;
    args.rd_part = b.rd->part;
    args.rd_out = b.rd->out;
    if (b.rd_done) *b.rd_done = 1u;
  }
  void* params[] = {&args};
  if (cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(kJitWarps * 32), params, smem,
                       (cudaStream_t)lc.stream) != cudaSuccess)
    return -1;
  return launched + 1;
}

int bs_jit_selftest(char* log, size_t cap) {
  // a run of a Toffoli, a CNOT, a controlled phase, a T and an X on 70 qubits
  Pass p;
  p.kind = PASS_FUSED;
  auto flip = [&](uint64_t c0, uint64_t c1, uint64_t t0, uint64_t t1) {
    FOp o;
    std::memset(&o, 0, sizeof(o));
    o.c[0] = c0;
    o.c[1] = c1;
    o.t[0] = t0;
    o.t[1] = t1;
    o.sbit = NO_SEL;
    o.ph = NO_PH;
    set_fop_kind(o);
    p.ops.push_back(o);
  };
  flip(0x3ull, 0ull, 0x4ull, 0ull);
  flip(0x8ull, 0ull, 0ull, 0x2ull);
  flip(0ull, 0ull, 0x10ull, 0ull);
  FOp ph;
  std::memset(&ph, 0, sizeof(ph));
  ph.c[0] = 0x21ull;
  ph.sbit = NO_SEL;
  ph.ph = 0;
  set_fop_kind(ph);
  p.ops.push_back(ph);
  p.phases.push_back(PhasePair{1.0, 0.0, 0.6, 0.8});
  FOp t;
  std::memset(&t, 0, sizeof(t));
  t.c[0] = 0x40ull;
  t.a0 = 1;
  t.sbit = NO_SEL;
  t.ph = NO_PH;
  set_fop_kind(t);
  p.ops.push_back(t);
  p.has_perm = true;
  p.has_phase = true;
  BsPass b;
  build_bitslice(p, 70, &b);
  const std::string src = make_source(b, 2, true, true, 32, nullptr);
  std::string msg;
  const std::string cubin = compile_cubin(src, 10, 3, &msg);
  if (log && cap) {
    std::snprintf(log, cap, "%s", cubin.empty() ? msg.c_str() : "ok");
  }
  return cubin.empty() ? 0 : 1;
}

}  // namespace sps
