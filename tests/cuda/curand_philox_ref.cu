// Test helper: cuRAND's own Philox4x32-10 (public device API) as an
// implementation independent of both the oracle and the AMH library.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void curand_philox_kernel(const uint4* ctr, const uint2* key, uint4* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_philox_ref(const unsigned* ctr, const unsigned* key, unsigned* out, int n) {
  uint4 *c = nullptr, *o = nullptr;
  uint2* k = nullptr;
  int rc = 0;
  if (cudaMalloc(&c, sizeof(uint4) * n) || cudaMalloc(&o, sizeof(uint4) * n) ||
      cudaMalloc(&k, sizeof(uint2) * n)) {
    rc = 1;
  } else if (cudaMemcpy(c, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice) ||
             cudaMemcpy(k, key, sizeof(uint2) * n, cudaMemcpyHostToDevice)) {
    rc = 2;
  } else {
    curand_philox_kernel<<<(n + 127) / 128, 128>>>(c, k, o, n);
    if (cudaMemcpy(out, o, sizeof(uint4) * n, cudaMemcpyDeviceToHost)) rc = 3;
  }
  cudaFree(c);
  cudaFree(o);
  cudaFree(k);
  return rc;
}
