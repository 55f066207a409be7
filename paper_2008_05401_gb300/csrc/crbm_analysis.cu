// Integrated autocorrelation time of many series on the device (the paper's
// comparison of samplers by the autocorrelation of the energy, Sec. III and
// Sec. IV).  Windowed estimator with Sokal's automatic window, per series
// x_0 .. x_{n-1}:
//   m = mean, G(t) = (1/n) sum_{s < n-t} (x_s - m)(x_{s+t} - m),
//   tau(W) = 1/2 + sum_{t=1}^{W} G(t)/G(0),  W = first W >= 1 with W >= c tau(W)
// (W <= n-1; a constant series gives tau = 1/2, W = 0).
// One CTA per series; each G(t) is a deterministic block sum, evaluated lag
// by lag until the window closes, so the work is O(n W) per series.
#include <mutex>

#include "crbm.h"
#include "crbm_device.cuh"
#include "crbm_kernels.h"

namespace crbm {

namespace {

constexpr int kTauThreads = 256;

// Series j of a time-major [n][n_series] array.
__global__ void __launch_bounds__(kTauThreads) tau_kernel(const double* __restrict__ x, int n_series, long long n,
                                                         double c, double* tau_out, long long* w_out) {
  __shared__ double sc[kTauThreads / 32];
  const int j = blockIdx.x;
  const int tid = threadIdx.x;
  const double* col = x + j;
  const long long ld = n_series;
  double s = 0.0;
  for (long long t = tid; t < n; t += kTauThreads) s += col[t * ld];
  const double m = block_sum(s, sc) / (double)n;
  double q = 0.0;
  for (long long t = tid; t < n; t += kTauThreads) {
    const double d = col[t * ld] - m;
    q = fma(d, d, q);
  }
  const double g0 = block_sum(q, sc) / (double)n;
  double tau = 0.5;
  long long W = 0;
  if (n >= 2 && g0 != 0.0) {
    W = n - 1;
    for (long long lag = 1; lag < n; ++lag) {
      double p = 0.0;
      for (long long t = tid; t < n - lag; t += kTauThreads) p = fma(col[t * ld] - m, col[(t + lag) * ld] - m, p);
      tau += (block_sum(p, sc) / (double)n) / g0;
      if ((double)lag >= c * tau) {
        W = lag;
        break;
      }
    }
  }
  if (tid == 0) {
    tau_out[j] = tau;
    w_out[j] = W;
  }
}

// Fixed device scratch of the no-allocation variant (crbm_autocorr_noalloc):
// tau[kMaxNoAllocSeries] FP64 followed by W[kMaxNoAllocSeries] int64, 256 KiB
// per device.  Each call's kernel writes every entry that the call copies
// back before the copy, so nothing in it has to start at zero.  All calls on
// a device share it: calls that overlap in time race.
constexpr int kMaxNoAllocSeries = CRBM_AUTOCORR_NOALLOC_MAX_SERIES;
static __device__ __align__(256) unsigned char g_tau_scratch[kMaxNoAllocSeries * 16];

}  // namespace

cudaError_t launch_tau(const double* x, int n_series, long long n, double c, double* tau, long long* w,
                       cudaStream_t st) {
  if (n_series == 0) return cudaSuccess;
  tau_kernel<<<n_series, kTauThreads, 0, st>>>(x, n_series, n, c, tau, w);
  return cudaGetLastError();
}

// Address of the scratch array on the current device, looked up once per
// device (cudaGetSymbolAddress; the first lookup on a device must not happen
// while a stream capture is in progress on it) and cached.
static cudaError_t tau_scratch(unsigned char** out) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static unsigned char* addr[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_tau_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = (unsigned char*)p;
  }
  *out = addr[dev];
  return cudaSuccess;
}

cudaError_t launch_tau_noalloc(const double* x, int n_series, long long n, double c, double* tau_host,
                               int64_t* w_host, cudaStream_t st) {
  if (n_series <= 0) return cudaSuccess;
  if (n_series > kMaxNoAllocSeries) return cudaErrorInvalidValue;
  unsigned char* base = nullptr;
  cudaError_t e = tau_scratch(&base);
  if (e != cudaSuccess) return e;
  double* d_tau = (double*)base;
  long long* d_w = (long long*)(base + (size_t)kMaxNoAllocSeries * 8);
  tau_kernel<<<n_series, kTauThreads, 0, st>>>(x, n_series, n, c, d_tau, d_w);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(tau_host, d_tau, (size_t)n_series * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w_host, d_w, (size_t)n_series * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

}  // namespace crbm
