// peaks.cu -- microbenchmarks of the units that bound the sweeps: FP32 FMA
// issue rate, MUFU square-root rate and L2 read bandwidth, on the device the
// benchmark runs on.  Used only to state the roofline denominators; no part
// of the sampler calls them.
#include <cuda_runtime.h>
#include <stdint.h>

#include "amh_peaks.h"

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

__global__ void __launch_bounds__(256) fma_kernel(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = threadIdx.x * 1e-3f + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == 1234.5f) out[blockIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(256) sqrt_kernel(float* out, int iters) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 2.f + threadIdx.x * 1e-3f + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int j = 0; j < kChains; ++j) {
        float y;
        asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[j]));
        x[j] = y + 1.5f;  // stays in [2, 4): one MUFU and one FADD per step
      }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == 1234.5f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) l2_read_kernel(const float4* __restrict__ buf, size_t n4,
                                                      int reps, float* out) {
  float acc = 0.f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      acc += v.x + v.y + v.z + v.w;
    }
  if (acc == 1234.5f) out[blockIdx.x] = acc;
}

float time_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

}  // namespace

extern "C" {

// Results: fp32_fma_per_s (FFMA instructions per second, whole GPU),
// mufu_sqrt_per_s (sqrt.approx per second), l2_read_bytes_per_s.  Returns 0
// or a CUDA error code.  Runs on the current device, synchronously.
int amh_measure_peaks(double* fp32_fma_per_s, double* mufu_sqrt_per_s,
                      double* l2_read_bytes_per_s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  float* out = nullptr;
  float4* buf = nullptr;
  const size_t bytes = (size_t)l2 / 2;  // resident in L2 after the first pass
  if ((e = cudaMalloc(&out, sizeof(float) * 65536)) != cudaSuccess) return (int)e;
  if ((e = cudaMalloc(&buf, bytes)) != cudaSuccess) {
    cudaFree(out);
    return (int)e;
  }
  cudaMemset(buf, 0, bytes);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  // FP32 FMA
  fma_kernel<<<blocks, threads>>>(out, 16, 0.999f, 1e-3f);
  cudaEventRecord(a);
  fma_kernel<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  *fp32_fma_per_s = (double)blocks * threads * iters * 16 * kChains / (time_ms(a, b) * 1e-3);
  // MUFU square root
  sqrt_kernel<<<blocks, threads>>>(out, 16);
  cudaEventRecord(a);
  sqrt_kernel<<<blocks, threads>>>(out, iters / 4);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  *mufu_sqrt_per_s = (double)blocks * threads * (iters / 4) * 16 * kChains / (time_ms(a, b) * 1e-3);
  // L2 reads of a buffer half the L2's size
  const size_t n4 = bytes / sizeof(float4);
  const int reps = 20;
  l2_read_kernel<<<blocks, threads>>>(buf, n4, 1, out);
  cudaEventRecord(a);
  l2_read_kernel<<<blocks, threads>>>(buf, n4, reps, out);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  *l2_read_bytes_per_s = (double)n4 * sizeof(float4) * reps / (time_ms(a, b) * 1e-3);
  e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  cudaFree(out);
  return (int)e;
}

}  // extern "C"
