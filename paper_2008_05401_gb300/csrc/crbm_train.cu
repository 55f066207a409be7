// The paper's CRBM trainer on the device (Sec. II, App. A, Algorithm 1):
// epochs of minibatch ADAM steps on the energy-matching loss
//   diff_i = t_i - F(x_i),  C = mean diff,  loss = mean (diff_i - C)^2,
//   d loss/d theta = (2/M) sum_i (diff_i - C) [ sum_ij sigma(a^f_ij) v_(i+a)(j+b),
//                                               sum_ij v_ij,  sum_ij sigma(a^f_ij) ]
// (the W, v_bias, h_bias components; sum_i (diff_i - C) = 0 removes C's own
// dependence on theta), then ADAM (Kingma & Ba 2014).  Everything is FP64.
//
// One CTA per training problem (the paper trains one CRBM per temperature):
// minibatch steps depend on each other through the parameters, so a problem
// runs its steps in order inside one CTA, with parameters, ADAM moments and
// the row-sum tables of the current filters in shared memory; independent
// problems fill the GPU side by side.  Per step: (1) row-sum tables of W,
// (2) one warp per sample: F (warp reductions) and the hidden probabilities
// sigma(a^f) kept in shared memory, then C and the loss, (3) one warp per
// parameter, lanes over (sample, site): the gradient, (4) ADAM.
#include <algorithm>

#include "crbm.h"
#include "crbm_device.cuh"
#include "crbm_kernels.h"

namespace crbm {

namespace {

constexpr int kTrainThreads = 512;
constexpr int kTrainWarps = kTrainThreads / 32;
constexpr size_t kSigBudget = 96 * 1024;   // shared memory for hidden probabilities

struct TrainParams {
  int n, batch;
  double lr, b1, b2, eps;
  crbm_train_problem pr[CRBM_TRAIN_MAX_PROBLEMS];
};

__device__ __forceinline__ double warp_sum64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Samples whose hidden probabilities fit the shared buffer at once.
__host__ __device__ inline int sig_capacity(int K, int N) {
  const size_t per = (size_t)K * N * 8;
  const size_t c = kSigBudget / per;
  return c < 1 ? 1 : (int)c;
}

// Hidden pre-activation of filter f at site (si, sj) of lattice v: h_bias^f
// plus one row-sum table entry per kernel row (window of k bits, periodic).
__device__ __forceinline__ double preact(const double* tab, double hb, int f, int k, int T, const int* codes) {
  double x = hb;
  for (int a = 0; a < k; ++a) x += tab[(f * k + a) * T + codes[a]];
  return x;
}

__device__ __forceinline__ void window_codes(const uint32_t* v, const int* wrap, int L, int k, int si, int sj,
                                             int (&codes)[kMaxk]) {
#pragma unroll
  for (int a = 0; a < kMaxk; ++a) {
    if (a >= k) break;
    const int r = wrap[si + a] * L;
    int c = 0;
    for (int b = 0; b < k; ++b) c |= (int)site_bit(v, r + wrap[sj + b]) << b;
    codes[a] = c;
  }
}

// Hidden probabilities sigma(a^f) of samples [i0, min(i1, i0 + cap)) into
// sig[(i - i0)][f][s] (the buffer holds cap samples); with F != nullptr also
// F(x_i) = -v_bias sum v - sum softplus(a^f) of every sample of [i0, i1).
// One warp per sample.
__device__ void hidden_pass(const uint32_t* vb, int Wd, const double* tab, const double* hbias, double vbias,
                            int K, int k, int T, int L, const int* wrap, int i0, int i1, int cap, double* sig,
                            double* F) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, N = L * L;
  for (int i = i0 + warp; i < i1; i += kTrainWarps) {
    const uint32_t* v = vb + i * Wd;
    const bool keep = i - i0 < cap;
    double sp = 0.0, ones = 0.0;
    for (int s = lane; s < N; s += 32) {
      const int si = s / L, sj = s - si * L;
      int codes[kMaxk];
      window_codes(v, wrap, L, k, si, sj, codes);
      for (int f = 0; f < K; ++f) {
        const double x = preact(tab, hbias[f], f, k, T, codes);
        const double e = exp(-fabs(x));
        sp += fmax(x, 0.0) + log1p(e);                           // softplus x
        if (keep) sig[((size_t)(i - i0) * K + f) * N + s] = (x >= 0.0 ? 1.0 : e) / (1.0 + e);   // sigma(x)
      }
      ones += (double)site_bit(v, s);
    }
    if (F) {
      sp = warp_sum64(sp);
      ones = warp_sum64(ones);
      if (lane == 0) F[i] = -vbias * ones - sp;
    }
  }
}

__global__ void __launch_bounds__(kTrainThreads, 1) train_epoch_kernel(const __grid_constant__ TrainParams p) {
  const crbm_train_problem& q = p.pr[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = q.K, k = q.k, L = q.L, N = L * L, T = 1 << k, Wd = (N + 31) / 32;
  const int nW = K * k * k, P = nW + 1 + K, nlut = K * k * T;
  const int M = p.batch, cap = sig_capacity(K, N);

  extern __shared__ __align__(16) unsigned char smem[];
  double* th = (double*)smem;              // P
  double* am = th + P;                      // P
  double* av = am + P;                      // P
  double* gr = av + P;                      // P: gradient of the minibatch
  double* tab = gr + P;                     // nlut
  double* Fs = tab + nlut;                  // M
  double* cw = Fs + M;                      // M: (2/M)(diff_i - C)
  double* sig = cw + M;                     // min(M, cap) * K * N
  uint32_t* vb = (uint32_t*)(sig + (size_t)min(M, cap) * K * N);   // M * Wd
  int* wrap = (int*)(vb + M * Wd);          // 2L: x -> x mod L

  for (int i = tid; i < P; i += kTrainThreads) {
    th[i] = q.theta[i];
    am[i] = q.adam_m[i];
    av[i] = q.adam_v[i];
  }
  for (int x = tid; x < 2 * L; x += kTrainThreads) wrap[x] = x < L ? x : x - L;
  long long t = *q.adam_t;
  __syncthreads();
  const int nb = (q.n_samples + M - 1) / M;
  for (int b = 0; b < nb; ++b) {
    const int b0 = b * M, Mb = min(M, q.n_samples - b0);
    // (1) row-sum tables of the current filters (bits summed in increasing b), samples
    for (int e = tid; e < nlut; e += kTrainThreads) {
      const int code = e % T, fa = e / T;
      double acc = 0.0;
      for (int bb = 0; bb < k; ++bb)
        if ((code >> bb) & 1) acc += th[fa * k + bb];
      tab[e] = acc;
    }
    for (int e = tid; e < Mb * Wd; e += kTrainThreads) {
      const int i = e / Wd, w = e - i * Wd;
      vb[e] = q.samples[(size_t)q.order[b0 + i] * Wd + w];
    }
    for (int i = tid; i < P; i += kTrainThreads) gr[i] = 0.0;
    __syncthreads();
    const double vbias = th[nW];
    const double* hbias = th + nW + 1;
    // (2) F of every sample (and the hidden probabilities of the first chunk)
    hidden_pass(vb, Wd, tab, hbias, vbias, K, k, T, L, wrap, 0, Mb, cap, sig, Fs);
    __syncthreads();
    if (tid == 0) {
      double C = 0.0;
      for (int i = 0; i < Mb; ++i) C += q.targets[q.order[b0 + i]] - Fs[i];
      C /= (double)Mb;
      double loss = 0.0;
      for (int i = 0; i < Mb; ++i) {
        const double d = q.targets[q.order[b0 + i]] - Fs[i] - C;
        loss += d * d;
        cw[i] = (2.0 / (double)Mb) * d;
      }
      if (q.losses) q.losses[b] = loss / (double)Mb;
    }
    __syncthreads();
    // (3) gradient: chunks of samples whose probabilities are in shared memory;
    // one warp per parameter, lanes over (sample, site), fixed reduction order
    for (int i0 = 0; i0 < Mb; i0 += cap) {
      const int i1 = min(Mb, i0 + cap);
      if (i0 > 0) {
        // the first pass kept the probabilities of the first chunk only: recompute this one
        __syncthreads();
        hidden_pass(vb, Wd, tab, hbias, vbias, K, k, T, L, wrap, i0, i1, cap, sig, nullptr);
        __syncthreads();
      }
      for (int pp = warp; pp < P; pp += kTrainWarps) {
        double acc = 0.0;
        if (pp < nW) {
          const int f = pp / (k * k), ab = pp - f * k * k, a = ab / k, bb = ab - a * k;
          for (int i = i0; i < i1; ++i) {
            const uint32_t* v = vb + i * Wd;
            const double* sg = sig + ((size_t)(i - i0) * K + f) * N;
            double part = 0.0;
            for (int s = lane; s < N; s += 32) {
              const int si = s / L, sj = s - si * L;
              if (site_bit(v, wrap[si + a] * L + wrap[sj + bb])) part += sg[s];
            }
            acc = fma(cw[i], part, acc);
          }
        } else if (pp == nW) {
          for (int i = i0; i < i1; ++i) {
            const uint32_t* v = vb + i * Wd;
            double part = 0.0;
            for (int s = lane; s < N; s += 32) part += (double)site_bit(v, s);
            acc = fma(cw[i], part, acc);
          }
        } else {
          const int f = pp - nW - 1;
          for (int i = i0; i < i1; ++i) {
            const double* sg = sig + ((size_t)(i - i0) * K + f) * N;
            double part = 0.0;
            for (int s = lane; s < N; s += 32) part += sg[s];
            acc = fma(cw[i], part, acc);
          }
        }
        acc = warp_sum64(acc);
        if (lane == 0) gr[pp] += acc;
      }
    }
    __syncthreads();
    // (4) ADAM
    t += 1;
    const double bc1 = 1.0 - pow(p.b1, (double)t), bc2 = 1.0 - pow(p.b2, (double)t);
    for (int pp = tid; pp < P; pp += kTrainThreads) {
      const double g = gr[pp];
      const double m = p.b1 * am[pp] + (1.0 - p.b1) * g;
      const double w = p.b2 * av[pp] + (1.0 - p.b2) * g * g;
      am[pp] = m;
      av[pp] = w;
      th[pp] = th[pp] - p.lr * (m / bc1) / (sqrt(w / bc2) + p.eps);
    }
    __syncthreads();
  }
  for (int i = tid; i < P; i += kTrainThreads) {
    q.theta[i] = th[i];
    q.adam_m[i] = am[i];
    q.adam_v[i] = av[i];
  }
  if (tid == 0) *q.adam_t = t;
}

}  // namespace

size_t train_smem_bytes(const crbm_train_problem& q, int batch) {
  const size_t N = (size_t)q.L * q.L, P = (size_t)q.K * q.k * q.k + 1 + q.K;
  const size_t nlut = (size_t)q.K * q.k * ((size_t)1 << q.k), Wd = (N + 31) / 32;
  const size_t chunk = (size_t)std::min(batch, sig_capacity(q.K, (int)N));
  return (4 * P + nlut + 2 * (size_t)batch + chunk * q.K * N) * 8 + (size_t)batch * Wd * 4 + 2 * (size_t)q.L * 4;
}

cudaError_t launch_train(const crbm_train_problem* pr, int n, int batch, double lr, double b1, double b2,
                         double eps, cudaStream_t st) {
  TrainParams p;
  p.n = n;
  p.batch = batch;
  p.lr = lr;
  p.b1 = b1;
  p.b2 = b2;
  p.eps = eps;
  size_t smem = 0;
  for (int i = 0; i < n; ++i) {
    p.pr[i] = pr[i];
    const size_t b = train_smem_bytes(pr[i], batch);
    if (b > smem) smem = b;
  }
  cudaError_t e = cudaFuncSetAttribute(train_epoch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  train_epoch_kernel<<<n, kTrainThreads, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace crbm
