// Small-state runs: one CTA applies a sequence of passes to a state of at most
// kSmallCap entries held in shared memory, so a chain of small passes costs one
// launch instead of one or two per pass.
//
// The passes run through the CTA engine (sps_cta_engine.cuh): gather-form
// branching (the insert-once rule of Sec. 3.1) and per-entry fused op lists.
#include <cuda_runtime.h>

#include <cstdint>

#include "sps_cta_engine.cuh"
#include "sps_device.cuh"
#include "sps_internal.h"

namespace sps {
namespace {

using namespace dev;

__device__ __forceinline__ cta::Bufs smem_bufs(unsigned char* base) {
  cta::Bufs s;
  s.lo = reinterpret_cast<uint64_t*>(base);
  s.hi = s.lo + kSmallCap;
  s.re = reinterpret_cast<double*>(s.hi + kSmallCap);
  s.im = s.re + kSmallCap;
  return s;
}

template <int KW>
__global__ void __launch_bounds__(kSmallThreads) k_small_run(Ctl* ctl, Bufs bufs,
                                                             const unsigned char* arena,
                                                             uint32_t pass_off, uint32_t npasses,
                                                             uint64_t capacity, uint32_t mg,
                                                             uint32_t serial_base,
                                                             uint32_t apply_serial,
                                                             unsigned long long* plog) {
  extern __shared__ __align__(16) unsigned char smem[];
  cta::Bufs A = smem_bufs(smem);
  cta::Bufs B = smem_bufs(smem + 32 * kSmallCap);
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
  uint64_t upd = 0;
  const uint32_t done = cta::run_passes<KW>(arena, passes, 0, npasses, A, B, n, cap, tab,
                                            kSmallTableSlots, warp_sums, &upd);
  if (done < npasses && threadIdx.x == 0)
    fail(ctl, SPS_ERR_CAPACITY, serial_base + passes[done].pass_serial,
         ((uint64_t)apply_serial << 32) | passes[done].fail_tag);
  // publish the state (after the last pass that succeeded) to the other buffer
  const SoA out = pick(bufs, cur ^ 1u);
  uint64_t mo0 = 0, mo1 = 0, ma0 = ~0ull, ma1 = ~0ull;   // OR / AND of the labels
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint64_t lo = A.lo[i], hi = A.hi[i];
    out.lo[i] = lo;
    if (KW == 2) out.hi[i] = hi;
    out.re[i] = A.re[i];
    out.im[i] = A.im[i];
    mo0 |= lo;
    mo1 |= hi;
    ma0 &= lo;
    ma1 &= hi;
  }
  merge_label_masks(ctl, mg_wr(mg), mo0, mo1, ma0, ma1);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    reset_label_masks(ctl, mg_rs(mg));
    ctl->nnz = n;
    ctl->cur = cur ^ 1u;
    ctl->updates += done < npasses ? upd - n : upd;
    if (plog) {
      plog[0] = n0;
      plog[1] = n;
    }
  }
}

}  // namespace

int launch_small_run(void* stream, int key_words, Ctl* ctl, Bufs bufs, const unsigned char* arena,
                     uint32_t pass_off, uint32_t npasses, uint64_t capacity, uint32_t mg,
                     uint32_t serial_base, uint32_t apply_serial, unsigned long long* plog) {
  const size_t smem = 64 * kSmallCap + 4 * (kSmallTableSlots + 33);
  if (key_words == 1) {
    cudaFuncSetAttribute(k_small_run<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_small_run<1><<<1, kSmallThreads, smem, (cudaStream_t)stream>>>(ctl, bufs, arena, pass_off,
                                                                      npasses, capacity, mg, serial_base,
                                                                      apply_serial, plog);
  } else {
    cudaFuncSetAttribute(k_small_run<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_small_run<2><<<1, kSmallThreads, smem, (cudaStream_t)stream>>>(ctl, bufs, arena, pass_off,
                                                                      npasses, capacity, mg, serial_base,
                                                                      apply_serial, plog);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace sps
