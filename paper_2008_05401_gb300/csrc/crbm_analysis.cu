// Integrated autocorrelation time of many series on the device (the paper's
// comparison of samplers by the autocorrelation of the energy, Sec. III and
// Sec. IV).  Windowed estimator with Sokal's automatic window, per series
// x_0 .. x_{n-1}:
//   m = mean, G(t) = (1/n) sum_{s < n-t} (x_s - m)(x_{s+t} - m),
//   tau(W) = 1/2 + sum_{t=1}^{W} G(t)/G(0),  W = first W >= 1 with W >= c tau(W)
// (W <= n-1; a constant series gives tau = 1/2, W = 0).
// One CTA per series; each G(t) is a deterministic block sum, evaluated lag
// by lag until the window closes, so the work is O(n W) per series.
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

}  // namespace

cudaError_t launch_tau(const double* x, int n_series, long long n, double c, double* tau, long long* w,
                       cudaStream_t st) {
  if (n_series == 0) return cudaSuccess;
  tau_kernel<<<n_series, kTauThreads, 0, st>>>(x, n_series, n, c, tau, w);
  return cudaGetLastError();
}

}  // namespace crbm
