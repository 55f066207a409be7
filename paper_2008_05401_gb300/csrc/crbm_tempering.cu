// Temperature-exchange step of the parallel-tempering correction (App. B.2,
// Fig. 8b) and of the local-update baselines with tempering.
//
// A ladder of physical chains x_i (target pi_i, temperature T_i fixed per
// slot).  In a tempering cycle the RBM chains have already made their
// proposal and been swapped with the physical chains (mode 2 of the fused
// kernel); one launch of this kernel then
//  1. exchanges neighbouring physical chains, pairs (0,1),(2,3),... on even
//     cycles and (1,2),(3,4),... on odd ones, with Eq. (B5) for (pi_i, pi_j):
//     log b = log pi_i(x_j) + log pi_j(x_i) - log pi_i(x_i) - log pi_j(x_j);
//     a state's weight at another temperature comes from its energy (Ising)
//     or from its cached spectrum eps (Kitaev): no new eigenvalue problem;
//  2. adds every physical chain's observables to its sums (and its energy to
//     the job's trace, if one is set).
// One warp per unit of at most two neighbouring chains (a pair of step 1, or
// a ladder end), so a unit needs no grid-wide synchronisation.  The cycle
// counter is the job's step counter plus an offset; the uniform of the pair
// (i, i+1) comes from tag kTagTemp of chain i.  Every value is FP64.
#include "crbm_device.cuh"
#include "crbm_kernels.h"

namespace crbm {

namespace {

struct PtParams {
  JobDev x;          // physical chains
  int step_offset;   // cycle counter = x's step counter + step_offset
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <typename E>
__device__ __forceinline__ void swap_rows(E* a, E* b, int n, int lane) {
  for (int w = lane; w < n; w += 32) {
    const E t = a[w];
    a[w] = b[w];
    b[w] = t;
  }
}

__device__ __forceinline__ void swap_scalar(double* a, double* b) {
  const double t = *a;
  *a = *b;
  *b = t;
}

__device__ __forceinline__ double log_uniform(const JobDev& x, uint32_t tag, uint32_t cycle, int i) {
  const uint4 w = philox4x32_10_rk(make_uint4(0u, tag, cycle, (uint32_t)(x.cid_base + (uint64_t)i)), x.rk);
  return log(((double)w.x + 0.5) * 0x1p-32);
}

// log pi_beta of a Kitaev state from its spectrum: sum_l log 2cosh(beta eps_l / 2)
__device__ __forceinline__ double kitaev_logpi_eps(const double* eps, int N, double beta, int lane) {
  double lp = 0.0, en = 0.0, cf = 0.0;
  for (int l = lane; l < N; l += 32) thermal_add(eps[l], beta, lp, en, cf);
  return warp_sum(lp);
}

// log pi, e, c_f (into the chain's current values) of Kitaev chain i at its temperature
__device__ __forceinline__ void kitaev_refresh(const JobDev& x, int i, int lane) {
  const double beta = 1.0 / x.T[i];
  double lp = 0.0, en = 0.0, cf = 0.0;
  const double* eps = x.eps + (size_t)i * x.N;
  for (int l = lane; l < x.N; l += 32) thermal_add(eps[l], beta, lp, en, cf);
  lp = warp_sum(lp);
  en = warp_sum(en);
  cf = warp_sum(cf);
  if (lane == 0) {
    x.logpi[i] = lp;
    x.Ephys[i] = en;
    double* ot = x.obs_t + (size_t)i * kNobs;
    ot[0] = en;
    ot[1] = en * en;
    ot[2] = cf;   // ot[3], the vison density, belongs to the lattice
  }
}

// Exchange every value that belongs to a lattice between slot i of job a and slot j of job b.
__device__ void swap_state(const JobDev& a, int i, const JobDev& b, int j, int lane) {
  const int Wd = a.Wd;
  swap_rows(a.bits + (size_t)i * Wd, b.bits + (size_t)j * Wd, Wd, lane);
  if (a.kind == kKitaev) swap_rows(a.eps + (size_t)i * a.N, b.eps + (size_t)j * a.N, a.N, lane);
  if (lane == 0) {
    swap_scalar(a.F + i, b.F + j);
    swap_scalar(a.Fb + i, b.Fb + j);
    swap_scalar(a.Lb + i, b.Lb + j);
    swap_scalar(a.logpi + i, b.logpi + j);
    swap_scalar(a.Ephys + i, b.Ephys + j);
    for (int o = 0; o < kNobs; ++o) swap_scalar(a.obs_t + (size_t)i * kNobs + o, b.obs_t + (size_t)j * kNobs + o);
  }
}

__global__ void __launch_bounds__(128) pt_exchange_kernel(const __grid_constant__ PtParams p) {
  const JobDev& x = p.x;
  const int lane = threadIdx.x & 31;
  const int u = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const unsigned long long cyc = *x.step + (long long)p.step_offset;
  const uint32_t cycle = (uint32_t)cyc;
  const int par = (int)(cycle & 1u);
  const int n = x.n_chains;
  const int lo = max(2 * u - par, 0), hi = min(2 * u + 2 - par, n);
  if (lo >= hi) return;
  // 1. temperature exchange of the pair (lo, lo + 1)
  if (hi - lo == 2) {
    const int i = lo, j = lo + 1;
    const double bi = 1.0 / x.T[i], bj = 1.0 / x.T[j];
    double lp_ij, lp_ji;   // log pi_i(x_j), log pi_j(x_i)
    if (x.kind == kKitaev) {
      lp_ij = kitaev_logpi_eps(x.eps + (size_t)j * x.N, x.N, bi, lane);
      lp_ji = kitaev_logpi_eps(x.eps + (size_t)i * x.N, x.N, bj, lane);
    } else {
      lp_ij = -bi * x.Ephys[j];
      lp_ji = -bj * x.Ephys[i];
    }
    int ex = 0;
    if (lane == 0) {
      const double log_b = lp_ij + lp_ji - x.logpi[i] - x.logpi[j];
      ex = log_uniform(x, kTagTemp, cycle, i) < log_b;
    }
    ex = __shfl_sync(kFull, ex, 0);
    if (ex) {
      swap_state(x, i, x, j, lane);
      __syncwarp();
      if (x.kind == kKitaev) {
        kitaev_refresh(x, i, lane);
        kitaev_refresh(x, j, lane);
      } else if (lane == 0) {
        // the energy and the observables belong to the lattice
        x.logpi[i] = -bi * x.Ephys[i];
        x.logpi[j] = -bj * x.Ephys[j];
      }
    }
  }
  __syncwarp();
  // 2. observables of the physical chains
  if (lane < (hi - lo) * kNobs) {
    const size_t e = (size_t)lo * kNobs + lane;
    x.obs[e] += x.obs_t[e];
  }
  if (lane < hi - lo) trace_store(x, lo + lane, cyc, x.Ephys[lo + lane]);
}

__global__ void pt_advance_kernel(unsigned long long* step) { *step += 1ull; }

}  // namespace

cudaError_t launch_pt_exchange(const JobDev& x, int step_offset, bool advance, cudaStream_t st) {
  if (x.n_chains == 0) return cudaSuccess;
  PtParams p;
  p.x = x;
  p.step_offset = step_offset;
  const int units = (x.n_chains + 2) / 2;     // most units over both parities
  const int warps = 4;
  pt_exchange_kernel<<<(units + warps - 1) / warps, 32 * warps, 0, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !advance) return e;
  pt_advance_kernel<<<1, 1, 0, st>>>(x.step);
  return cudaGetLastError();
}

}  // namespace crbm
