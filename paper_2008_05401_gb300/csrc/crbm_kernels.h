// Host-side entry points into the kernels of crbm_kernels.cu.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace crbm {
struct LaunchParams;
struct JobDev;

// Compiled specialisation (KC, kC) serving a filter bank of K filters k x k
// (0 = runtime values).
void specialisation(int K, int k, int& KC, int& kC);
// Dynamic shared memory of one CTA of the fused kernel (ncls kernel classes
// in the tables: 1 for a CRBM, 2 edge + 1 for an LCRBM).
size_t smem_bytes(int kind, int prec, int L, int K, int k, int nc, int KC, int ncls = 1);
// Threads per CTA of an Ising launch: 256 (a Kitaev launch takes the largest
// group size of its jobs, see kitaev_group_threads).
int threads_for(int kind, int max_N);
// Default threads of one Kitaev chain's group (its eigen-stage): 32 up to 16
// cells, 64 up to 64, 128 up to 100, else 256 (measured: small groups wait
// less at the eigen-stage barriers).
int kitaev_group_threads(int N);
// Launch the fused kernel: grid = total tiles of all jobs in p (one filter shape per launch);
// generic: use the runtime-shape variant even where a specialisation exists (LCRBM jobs);
// multi: Kitaev proposals (mode 0) in 256-thread CTAs holding several chain groups.
cudaError_t launch_step(int kind, int prec, int K, int k, int nt, const LaunchParams& p, int grid, size_t smem,
                        cudaStream_t st, bool generic = false, bool multi = false);
// Raise the dynamic shared-memory limit of every fused-kernel instantiation.
cudaError_t set_smem_limits(size_t bytes);
// Tensor-core form of the proposal kernel (crbm_step_tc.cu): Ising kind, mixed
// precision, L = 128 (one chain per CTA tile), 64 (two), 32 (four) or 16
// (eight), K <= 4, k <= 5.  One persistent launch serves jobs of every side:
// grid CTAs take the p.total_items tiles from the counter p.queue (zero at
// launch; cleared again after it).
bool tc_supported(int kind, int prec, int L, int K, int k);
int tc_chains_per_cta(int L);
size_t tc_smem_bytes(int L, int K, int k);
cudaError_t launch_tc(const LaunchParams& p, int grid, size_t smem, cudaStream_t st);
cudaError_t tc_set_smem_limit();
// One CTA waiting on an mbarrier with the tensor-core pipeline's bounded wait
// (arrive = 0: nothing arrives; after `limit` cycles *err = timeout).
cudaError_t launch_wait_probe(long long limit, int arrive, int* err, cudaStream_t st);
// Random initial lattices (init tag of the stream).
cudaError_t launch_random_init(uint32_t* bits, int n_chains, int N, int Wd, uint64_t seed,
                               uint64_t cid_base, cudaStream_t st);
// Neighbour temperature exchange of one cycle (crbm_tempering.cu) on job x;
// the cycle counter is x's step counter + step_offset; `advance` then adds
// one to x's step counter.
cudaError_t launch_pt_exchange(const JobDev& x, int step_offset, bool advance, cudaStream_t st);
// Integrated autocorrelation time of every column of a time-major
// [n][n_series] device array (crbm_analysis.cu); tau and w are device arrays.
cudaError_t launch_tau(const double* x, int n_series, long long n, double c, double* tau, long long* w,
                       cudaStream_t st);
// The same into a fixed device scratch array (no device allocation), results
// copied to the host arrays; returns after the copies.  n_series must not
// exceed CRBM_AUTOCORR_NOALLOC_MAX_SERIES.
cudaError_t launch_tau_noalloc(const double* x, int n_series, long long n, double c, double* tau_host,
                               int64_t* w_host, cudaStream_t st);
// Trainer (crbm_train.cu): one epoch of each of n <= CRBM_TRAIN_MAX_PROBLEMS
// problems (crbm_train_problem is declared in crbm.h).
}  // namespace crbm
#include "crbm.h"
namespace crbm {
size_t train_smem_bytes(const crbm_train_problem& q, int batch);
// Measured FP32 / FP64 FMA throughput of `device` (crbm_analysis.cu).
cudaError_t probe_fma_peaks(int device, double* fp32_tflops, double* fp64_tflops, cudaStream_t st);
cudaError_t launch_train(const crbm_train_problem* pr, int n, int batch, double lr, double b1, double b2,
                         double eps, cudaStream_t st);
}  // namespace crbm
