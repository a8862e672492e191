// Issue-rate probe for the units the sparse-state kernels lean on: FP64 fused
// multiply-add (amplitude products), FP32 fused multiply-add, three-input logic
// (the bit-sliced op walk and transposes) and 32-bit integer multiply-add
// (fixed-point phase products). Each thread runs 8 independent dependent
// chains written as inline PTX, so the compiler can neither fold nor drop them;
// rates are chain operations per second over a timed launch (CUDA events).
#include <cuda_runtime.h>

#include <cstdint>

#include "sps.h"

namespace {

constexpr int kChains = 8;
constexpr int kIter = 2048;

template <int K>
__global__ void __launch_bounds__(256) k_probe(uint64_t* out, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t acc = 0;
  if (K == 0) {   // FP64 fma
    double a[kChains];
    for (int c = 0; c < kChains; ++c) a[c] = 1.0 + 1e-9 * (tid + c + seed);
    const double m = 0.999999999, b = 1e-9;
    for (int i = 0; i < kIter; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[c]) : "d"(m), "d"(b));
    for (int c = 0; c < kChains; ++c) acc += (uint64_t)__double_as_longlong(a[c]);
  } else if (K == 1) {   // FP32 fma
    float a[kChains];
    for (int c = 0; c < kChains; ++c) a[c] = 1.0f + 1e-6f * (float)(tid % 97 + c + seed);
    const float m = 0.9999f, b = 1e-4f;
    for (int i = 0; i < kIter; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(m), "f"(b));
    for (int c = 0; c < kChains; ++c) acc += __float_as_uint(a[c]);
  } else if (K == 2) {   // three-input logic
    uint32_t a[kChains];
    for (int c = 0; c < kChains; ++c) a[c] = tid * 2654435761u + c + seed;
    const uint32_t b = 0x9E3779B9u ^ seed, d = 0x7F4A7C15u;
    for (int i = 0; i < kIter; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c)
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[c]) : "r"(b), "r"(d));
    for (int c = 0; c < kChains; ++c) acc += a[c];
  } else {   // 32-bit integer multiply-add
    uint32_t a[kChains];
    for (int c = 0; c < kChains; ++c) a[c] = tid + c + seed;
    const uint32_t m = 0x9E3779B1u, b = 12345u;
    for (int i = 0; i < kIter; ++i)
#pragma unroll
      for (int c = 0; c < kChains; ++c)
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(m), "r"(b));
    for (int c = 0; c < kChains; ++c) acc += a[c];
  }
  out[tid] = acc;
}

template <int K>
float time_probe(uint64_t* out, int blocks, cudaStream_t st) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.f;
  }
  k_probe<K><<<blocks, 256, 0, st>>>(out, 1u);   // warm-up
  cudaEventRecord(e0, st);
  for (int r = 0; r < 3; ++r) k_probe<K><<<blocks, 256, 0, st>>>(out, (uint32_t)r);
  cudaEventRecord(e1, st);
  float ms = -1.f;
  if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / 3.f;
}

}  // namespace

extern "C" sps_status sps_device_rates(double rates[4]) {
  if (!rates) return SPS_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return SPS_ERR_NO_DEVICE;
  }
  const int blocks = sms * 8;
  const size_t threads = (size_t)blocks * 256;
  uint64_t* out = nullptr;
  if (cudaMalloc(&out, threads * sizeof(uint64_t)) != cudaSuccess) {
    cudaGetLastError();
    return SPS_ERR_OOM;
  }
  cudaStream_t st = nullptr;
  const double ops = (double)threads * kChains * kIter;
  const float t[4] = {time_probe<0>(out, blocks, st), time_probe<1>(out, blocks, st),
                      time_probe<2>(out, blocks, st), time_probe<3>(out, blocks, st)};
  const cudaError_t e = cudaDeviceSynchronize();
  cudaFree(out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SPS_ERR_CUDA;
  }
  for (int k = 0; k < 4; ++k) rates[k] = t[k] > 0.f ? ops / (t[k] * 1e-3) : 0.0;
  return SPS_OK;
}
