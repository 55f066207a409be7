// Host-facing helpers of the fused kernel: shared-memory sizing, dispatch to
// the compiled (kind, precision, K, k) variants, random initial lattices.
#include "crbm_step.cuh"

namespace crbm {

size_t smem_bytes(int kind, int prec, int L, int K, int k, int nc, int KC, int ncls) {
  const size_t N = (size_t)L * L, P = (N + 31) / 32 + 1, nlut = (size_t)ncls * K * k * ((size_t)1 << k);
  const size_t nq = (size_t)k << k;
  size_t b = (prec == kFP64) ? 2 * align16(nlut * 8)
             : (KC == 4 ? 3 * align16(nq * 16 * 8) + align16(nlut * 4) : 4 * align16(nlut * 4));
  b += align16(nc * sizeof(ChainSm));
  b += align16(64 * 8);
  if (kind == kKitaev) b += (size_t)nc * kitaev_work_bytes((int)N);
  b += align16((size_t)nc * (2 + K) * P * 4);
  return b;
}


// v_ij = [u < 1/2] from the stream's init tag: one thread per packed word.
__global__ void random_init_kernel(uint32_t* bits, int n_chains, int N, int Wd, uint64_t seed,
                                   uint64_t cid_base) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_chains * Wd) return;
  const int c = (int)(idx / Wd), w = (int)(idx - (long long)c * Wd);
  const uint32_t cid = (uint32_t)(cid_base + (uint64_t)c);
  uint32_t out = 0;
  for (int q8 = 0; q8 < 8; ++q8) {
    const int q = w * 8 + q8;
    if (4 * q >= N) break;
    const uint4 r = philox4x32_10(make_uint4((uint32_t)q, kTagInit, 0u, cid), (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
    for (int t = 0; t < 4; ++t)
      if (4 * q + t < N && pick(r, t) < 0x80000000u) out |= 1u << (4 * q8 + t);
  }
  bits[idx] = out;
}

cudaError_t launch_kIsing_kFP64_256(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kIsing_kFP64_256(size_t);
cudaError_t launch_kIsing_kMixed_256(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kIsing_kMixed_256(size_t);
cudaError_t launch_kKitaev_kFP64_256(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kKitaev_kFP64_256(size_t);
cudaError_t launch_kKitaev_kFP64_128(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kKitaev_kFP64_128(size_t);
cudaError_t launch_kKitaev_kFP64_64(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kKitaev_kFP64_64(size_t);
cudaError_t launch_kKitaev_kFP64_32(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kKitaev_kFP64_32(size_t);
cudaError_t launch_kKitaev_kMixed_256(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kKitaev_kMixed_256(size_t);
cudaError_t launch_kKitaev_kMixed_128(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kKitaev_kMixed_128(size_t);
cudaError_t launch_kKitaev_kMixed_64(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kKitaev_kMixed_64(size_t);
cudaError_t launch_kKitaev_kMixed_32(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kKitaev_kMixed_32(size_t);
cudaError_t launch_kKitaev_kFP64_256_multi(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kKitaev_kFP64_256_multi(size_t);
cudaError_t launch_kKitaev_kMixed_256_multi(int, int, const LaunchParams&, int, size_t, cudaStream_t);
cudaError_t limit_kKitaev_kMixed_256_multi(size_t);

void specialisation(int K, int k, int& KC, int& kC) {
  KC = 0;
  kC = 0;
  if (K == 4 && (k == 5 || k == 3)) {
    KC = 4;
    kC = k;
  }
}

// Ising jobs run in CTAs of 256 threads.  A Kitaev chain is run by a thread
// group of its own (kitaev_group_threads or its tuned size); a launch of
// Kitaev jobs takes CTAs of the largest group size among them, so jobs of
// every lattice side share one launch, several small chains per CTA.
int threads_for(int, int) { return 256; }

// Threads of a Kitaev chain's group, measured on the Kitaev workloads when
// they were CTA sizes: 32 up to 16 cells, 64 up to 64, 128 up to 100 and 256
// above (the reduction's per-column barriers cost less in small groups).
int kitaev_group_threads(int N) { return N <= 16 ? 32 : (N <= 64 ? 64 : (N <= 100 ? 128 : 256)); }

cudaError_t launch_step(int kind, int prec, int K, int k, int nt, const LaunchParams& p, int grid, size_t smem,
                        cudaStream_t st, bool generic, bool multi) {
  int KC, kC;
  specialisation(K, k, KC, kC);
  if (generic) KC = kC = 0;
  if (multi)
    return prec == kFP64 ? launch_kKitaev_kFP64_256_multi(KC, kC, p, grid, smem, st)
                         : launch_kKitaev_kMixed_256_multi(KC, kC, p, grid, smem, st);
  if (kind == kIsing)
    return prec == kFP64 ? launch_kIsing_kFP64_256(KC, kC, p, grid, smem, st)
                         : launch_kIsing_kMixed_256(KC, kC, p, grid, smem, st);
  if (prec == kFP64) {
    switch (nt) {
      case 32: return launch_kKitaev_kFP64_32(KC, kC, p, grid, smem, st);
      case 64: return launch_kKitaev_kFP64_64(KC, kC, p, grid, smem, st);
      case 128: return launch_kKitaev_kFP64_128(KC, kC, p, grid, smem, st);
      default: return launch_kKitaev_kFP64_256(KC, kC, p, grid, smem, st);
    }
  }
  switch (nt) {
    case 32: return launch_kKitaev_kMixed_32(KC, kC, p, grid, smem, st);
    case 64: return launch_kKitaev_kMixed_64(KC, kC, p, grid, smem, st);
    case 128: return launch_kKitaev_kMixed_128(KC, kC, p, grid, smem, st);
    default: return launch_kKitaev_kMixed_256(KC, kC, p, grid, smem, st);
  }
}

cudaError_t set_smem_limits(size_t bytes) {
  cudaError_t e = cudaSuccess;
  for (cudaError_t (*f)(size_t) : {limit_kIsing_kFP64_256, limit_kIsing_kMixed_256, limit_kKitaev_kFP64_256,
                                   limit_kKitaev_kFP64_128, limit_kKitaev_kFP64_64, limit_kKitaev_kFP64_32,
                                   limit_kKitaev_kMixed_256, limit_kKitaev_kMixed_128, limit_kKitaev_kMixed_64,
                                   limit_kKitaev_kMixed_32, limit_kKitaev_kFP64_256_multi,
                                   limit_kKitaev_kMixed_256_multi})
    if (e == cudaSuccess) e = f(bytes);
  return e;
}

cudaError_t launch_random_init(uint32_t* bits, int n_chains, int N, int Wd, uint64_t seed,
                               uint64_t cid_base, cudaStream_t st) {
  const long long total = (long long)n_chains * Wd;
  if (total == 0) return cudaSuccess;
  const int blocks = (int)((total + 255) / 256);
  random_init_kernel<<<blocks, 256, 0, st>>>(bits, n_chains, N, Wd, seed, cid_base);
  return cudaGetLastError();
}

}  // namespace crbm
