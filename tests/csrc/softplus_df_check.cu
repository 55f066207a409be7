// Test helper: the library's double-FP32 softplus (crbm_df64.cuh) evaluated
// on given df64 arguments, for tests/test_gpu_softplus_df.py.
#include <cuda_runtime.h>

#include "crbm_df64.cuh"

using namespace crbm;

static __global__ void eval_kernel(const float* hi, const float* lo, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const df r = softplus_df({hi[i], lo[i]});
  out[i] = (double)r.hi + (double)r.lo;
}

// out[i] = softplus_df(hi[i] + lo[i]) for host arrays of n entries; 0 on success.
extern "C" int softplus_df_eval(const float* hi, const float* lo, double* out, int n) {
  float *dh = nullptr, *dl = nullptr;
  double* dout = nullptr;
  int rc = 1;
  if (cudaMalloc(&dh, n * sizeof(float)) == cudaSuccess && cudaMalloc(&dl, n * sizeof(float)) == cudaSuccess &&
      cudaMalloc(&dout, n * sizeof(double)) == cudaSuccess &&
      cudaMemcpy(dh, hi, n * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
      cudaMemcpy(dl, lo, n * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess) {
    eval_kernel<<<(n + 255) / 256, 256>>>(dh, dl, dout, n);
    if (cudaGetLastError() == cudaSuccess &&
        cudaMemcpy(out, dout, n * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess)
      rc = 0;
  }
  cudaFree(dh);
  cudaFree(dl);
  cudaFree(dout);
  return rc;
}
