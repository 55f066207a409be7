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
// (2) F of every sample of the minibatch (block reductions), C and the loss,
// (3) per sample the hidden probabilities sigma(a^f) in shared memory, then
// one thread per parameter accumulates its gradient component, (4) ADAM.
#include "crbm.h"
#include "crbm_device.cuh"
#include "crbm_kernels.h"

namespace crbm {

namespace {

constexpr int kTrainThreads = 256;

struct TrainParams {
  int n, batch;
  double lr, b1, b2, eps;
  crbm_train_problem pr[CRBM_TRAIN_MAX_PROBLEMS];
};

__device__ __forceinline__ double sigmoid64(double x) { return 1.0 / (1.0 + exp(-x)); }

// Hidden pre-activation of filter f at site (i, j): h_bias^f plus the row-sum
// table entries of the k kernel rows (codes of the k-bit windows).
__device__ __forceinline__ double preact(const double* tab, double hb, int f, int k, int T, const int* codes) {
  double x = hb;
  for (int a = 0; a < k; ++a) x += tab[(f * k + a) * T + codes[a]];
  return x;
}

__device__ __forceinline__ void window_codes(const uint32_t* v, int L, int k, int i, int j, int* codes) {
  for (int a = 0; a < k; ++a) {
    const int r = (i + a) % L;
    int c = 0;
    for (int b = 0; b < k; ++b) c |= (int)site_bit(v, r * L + (j + b) % L) << b;
    codes[a] = c;
  }
}

__global__ void __launch_bounds__(kTrainThreads) train_epoch_kernel(const __grid_constant__ TrainParams p) {
  const crbm_train_problem& q = p.pr[blockIdx.x];
  const int tid = threadIdx.x;
  const int K = q.K, k = q.k, L = q.L, N = L * L, T = 1 << k, Wd = (N + 31) / 32;
  const int nW = K * k * k, P = nW + 1 + K, nlut = K * k * T;
  const int M = p.batch;

  extern __shared__ __align__(16) unsigned char smem[];
  double* th = (double*)smem;              // P
  double* am = th + P;                      // P
  double* av = am + P;                      // P
  double* tab = av + P;                     // nlut
  double* sig = tab + nlut;                 // K * N
  double* Fs = sig + (size_t)K * N;         // M
  double* cw = Fs + M;                      // M: (2/M)(diff_i - C)
  double* sc = cw + M;                      // 64: reduction scratch
  uint32_t* vb = (uint32_t*)(sc + 64);      // M * Wd

  for (int i = tid; i < P; i += kTrainThreads) {
    th[i] = q.theta[i];
    am[i] = q.adam_m[i];
    av[i] = q.adam_v[i];
  }
  long long t = *q.adam_t;
  __syncthreads();
  const int nb = (q.n_samples + M - 1) / M;
  for (int b = 0; b < nb; ++b) {
    const int b0 = b * M, Mb = min(M, q.n_samples - b0);
    // (1) row-sum tables of the current filters, bits summed in increasing b
    for (int e = tid; e < nlut; e += kTrainThreads) {
      const int code = e % T, fa = e / T;
      double s = 0.0;
      for (int bb = 0; bb < k; ++bb)
        if ((code >> bb) & 1) s += th[fa * k + bb];
      tab[e] = s;
    }
    for (int e = tid; e < Mb * Wd; e += kTrainThreads) {
      const int i = e / Wd, w = e - i * Wd;
      vb[e] = q.samples[(size_t)q.order[b0 + i] * Wd + w];
    }
    __syncthreads();
    const double vbias = th[nW];
    // (2) F(x_i) = -v_bias sum v - sum_{f,ij} softplus(a^f_ij)
    for (int i = 0; i < Mb; ++i) {
      const uint32_t* v = vb + i * Wd;
      double sp = 0.0, ones = 0.0;
      for (int s = tid; s < N; s += kTrainThreads) {
        const int si = s / L, sj = s - si * L;
        int codes[kMaxk];
        window_codes(v, L, k, si, sj, codes);
        for (int f = 0; f < K; ++f) sp += softplus64(preact(tab, th[nW + 1 + f], f, k, T, codes));
        ones += (double)site_bit(v, s);
      }
      sp = block_sum(sp, sc);
      ones = block_sum(ones, sc);
      if (tid == 0) Fs[i] = -vbias * ones - sp;
    }
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
    // (3) gradient, one thread per parameter, samples in minibatch order
    double g0 = 0.0, g1 = 0.0;               // this thread's components p = tid, tid + 256
    for (int i = 0; i < Mb; ++i) {
      const uint32_t* v = vb + i * Wd;
      for (int s = tid; s < N; s += kTrainThreads) {
        const int si = s / L, sj = s - si * L;
        int codes[kMaxk];
        window_codes(v, L, k, si, sj, codes);
        for (int f = 0; f < K; ++f) sig[f * N + s] = sigmoid64(preact(tab, th[nW + 1 + f], f, k, T, codes));
      }
      __syncthreads();
      const double c = cw[i];
      for (int r = 0; r < 2; ++r) {
        const int pp = tid + r * kTrainThreads;
        if (pp >= P) break;
        double acc = 0.0;
        if (pp < nW) {
          const int f = pp / (k * k), ab = pp - f * k * k, a = ab / k, bb = ab - a * k;
          for (int s = 0; s < N; ++s) {
            const int si = s / L, sj = s - si * L;
            if (site_bit(v, ((si + a) % L) * L + (sj + bb) % L)) acc += sig[f * N + s];
          }
        } else if (pp == nW) {
          for (int s = 0; s < N; ++s) acc += (double)site_bit(v, s);
        } else {
          const int f = pp - nW - 1;
          for (int s = 0; s < N; ++s) acc += sig[f * N + s];
        }
        if (r == 0) g0 = fma(c, acc, g0);
        else g1 = fma(c, acc, g1);
      }
      __syncthreads();
    }
    // (4) ADAM
    t += 1;
    const double bc1 = 1.0 - pow(p.b1, (double)t), bc2 = 1.0 - pow(p.b2, (double)t);
    for (int r = 0; r < 2; ++r) {
      const int pp = tid + r * kTrainThreads;
      if (pp >= P) break;
      const double g = r == 0 ? g0 : g1;
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
  return (3 * P + nlut + q.K * N + 2 * (size_t)batch + 64) * 8 + (size_t)batch * Wd * 4;
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
