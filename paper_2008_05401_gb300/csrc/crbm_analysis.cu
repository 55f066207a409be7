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

// ------------------------------------------------------------------ peak probes
// FMA throughput of the FP32 and FP64 pipes: every thread runs 8 independent
// dependency chains of fused multiply-adds (enough to hide the pipe latency),
// the grid fills every SM several times over; a checksum of all chains is
// stored so that the compiler keeps the work.
namespace crbm {
namespace {

template <typename R>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, R a, R b, R* sink) {
  R x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (R)(threadIdx.x + c) * (R)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = x[c] * a + b;
  }
  R s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// Measured FMA rate (TFLOP/s, 2 flops per FMA) of one precision on the current device.
template <typename R>
static cudaError_t probe_one(int sms, R* sink, cudaStream_t st, double* tflops) {
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(R) == 8 ? 256 : 4096;     // about a second of FP64, a quarter of FP32
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  fma_probe_kernel<R><<<blocks, threads, 0, st>>>(iters / 8, (R)0.999, (R)1e-4, sink);   // warm-up
  cudaEventRecord(e0, st);
  fma_probe_kernel<R><<<blocks, threads, 0, st>>>(iters, (R)0.999, (R)1e-4, sink);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / ((double)ms * 1e-3) / 1e12;
  return cudaGetLastError();
}

cudaError_t probe_fma_peaks(int device, double* fp32_tflops, double* fp64_tflops, cudaStream_t st) {
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  const size_t n = (size_t)sms * 8 * 256;
  double* sink = nullptr;
  e = cudaMalloc(&sink, n * sizeof(double));
  if (e != cudaSuccess) return e;
  e = probe_one<float>(sms, (float*)sink, st, fp32_tflops);
  if (e == cudaSuccess) e = probe_one<double>(sms, sink, st, fp64_tflops);
  cudaStreamSynchronize(st);
  cudaFree(sink);
  return e;
}

}  // namespace crbm
