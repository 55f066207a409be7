// Exhaustive check of the special-function approximations the mixed-precision
// path certifies its margins with (ex2, rcp, lg2 in crbm_device.cuh), and of
// the FP32 conditional sigma(x) they compose: every float of the tested range
// is evaluated and the largest error against an FP64 reference is returned.
// Test-suite helper, not part of the library.
#include <cstdint>
#include <cstring>
#include "crbm_device.cuh"

namespace {
__device__ unsigned long long g_max[4];

__device__ void fold(int slot, double err) {
  // non-negative doubles order like their bit patterns
  atomicMax(&g_max[slot], (unsigned long long)__double_as_longlong(err));
}

// all floats with bit patterns in [b0, b1)
__global__ void sweep(int which, uint32_t b0, uint32_t b1) {
  double worst = 0.0;
  for (uint64_t i = b0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b1;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const float x = __uint_as_float((uint32_t)i);
    double err;
    if (which == 0) {
      const double ref = exp2((double)x);
      err = fabs((double)crbm::ex2_approx(x) - ref) / ref;
    } else if (which == 1) {
      const double ref = 1.0 / (double)x;
      err = fabs((double)crbm::rcp_approx(x) - ref) / ref;
    } else if (which == 2) {
      err = fabs((double)crbm::lg2_approx(x) - log2((double)x));
    } else {
      const double ref = 1.0 / (1.0 + exp(-(double)x));
      err = fabs((double)crbm::sigmoid32(x) - ref) / ref;
    }
    worst = fmax(worst, err);
  }
  fold(which, worst);
}
}  // namespace

extern "C" int sfu_max_error(int which, uint32_t b0, uint32_t b1, double* out) {
  if (which < 0 || which > 3) return -4;
  unsigned long long zero[4] = {0, 0, 0, 0};
  if (cudaMemcpyToSymbol(g_max, zero, sizeof zero) != cudaSuccess) return -1;
  sweep<<<1216, 256>>>(which, b0, b1);
  if (cudaDeviceSynchronize() != cudaSuccess) return -2;
  unsigned long long h[4];
  if (cudaMemcpyFromSymbol(h, g_max, sizeof h) != cudaSuccess) return -3;
  std::memcpy(out, &h[which], sizeof(double));
  return 0;
}
