// Test helper: the tensor-core kernel's FP32 log u of an MH draw
// (log_u32, crbm_device.cuh) evaluated on given 32-bit draws, for
// tests/test_gpu_log_u32.py.
#include <cuda_runtime.h>

#include "crbm_device.cuh"

using namespace crbm;

static __global__ void eval_kernel(const uint32_t* w, float* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = log_u32(w[i]);
}

// out[i] = log_u32(w[i]) for host arrays of n entries; 0 on success.
extern "C" int log_u32_eval(const uint32_t* w, float* out, int n) {
  uint32_t* dw = nullptr;
  float* dout = nullptr;
  int rc = 1;
  if (cudaMalloc(&dw, n * sizeof(uint32_t)) == cudaSuccess && cudaMalloc(&dout, n * sizeof(float)) == cudaSuccess &&
      cudaMemcpy(dw, w, n * sizeof(uint32_t), cudaMemcpyHostToDevice) == cudaSuccess) {
    eval_kernel<<<(n + 255) / 256, 256>>>(dw, dout, n);
    if (cudaGetLastError() == cudaSuccess && cudaMemcpy(out, dout, n * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess)
      rc = 0;
  }
  cudaFree(dw);
  cudaFree(dout);
  return rc;
}
