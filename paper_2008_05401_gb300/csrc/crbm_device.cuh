// Device-side building blocks of the CRBM proposal + Metropolis-Hastings step.
//
// Method: arXiv:2008.05401.  CRBM joint/free energy (Sec. II, Eqs. 12-13),
// Gibbs conditionals (App. B.1, Eqs. B1-B4), acceptance (App. B.2, Eq. B5),
// Ising energy (Sec. III, Eq. 14), Kitaev Majorana log-weight (Sec. IV,
// Eq. 16 and the free energy that follows it).
//
// Data layout in shared memory (one chain):
//   plane = ceil(L*L/32) + 1 uint32 words, site n = i*L + j is bit n%32 of
//   word n/32, the extra word is padding read (and masked) by row extraction.
//   Per chain: plane[0], plane[1] (current / proposed lattice, swapped on
//   accept), K hidden planes.
// Work unit: a block of 4 consecutive sites n = 4q..4q+3.  One Philox call
// gives the 4 uniforms of a unit for one tag, so a unit is owned by one thread.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace crbm {

constexpr int kMaxK = 8;
constexpr int kMaxk = 7;
constexpr int kMaxJobs = 16;
constexpr int kNobs = 4;
constexpr uint32_t kTagAcc = 0xFFFFFFFEu;
constexpr uint32_t kTagInit = 0xFFFFFFFFu;
constexpr uint32_t kTagSwap = 0xFFFFFFFDu;   // tempering: physical <-> RBM exchange
constexpr uint32_t kTagTemp = 0xFFFFFFFCu;   // tempering: neighbour temperature exchange
constexpr uint32_t kTagLocal = 0xFFFFFFFBu;  // local-update Metropolis sweeps
constexpr int kIsing = 0;
constexpr int kKitaev = 1;
constexpr int kFP64 = 0;
constexpr int kMixed = 1;
// Threads per CTA of the fused kernel and the CTAs per SM its register budget
// is sized for (compile-time; the defaults were chosen by measurement).
#ifndef CRBM_THREADS
#define CRBM_THREADS 256
#endif
#ifndef CRBM_MIN_BLOCKS
#define CRBM_MIN_BLOCKS 2
#endif
constexpr int kThreads = CRBM_THREADS;
constexpr unsigned kFull = 0xffffffffu;

enum DevErr : int { kErrNone = 0, kErrConfig = 1, kErrTimeout = 2 };

// Everything a kernel needs about one job; passed by value in the launch
// parameters.  Pointers into the job's caller-owned device memory.
struct JobDev {
  int kind, L, N, Wd, P, K, k, n_chains, nc;
  int lc_edge;                  // > 0: LCRBM with lc_edge unshared kernels per side; lattice open along j
  int ncls;                     // kernel classes in the tables: 2 lc_edge + 1, or 1
  int nhex;                     // Kitaev hexagons: N, or L (L-1) with open columns
  double vb;
  double hb[kMaxK];
  double J[3];
  float vb32;
  float hb32[kMaxK], hb_hi[kMaxK], hb_lo[kMaxK];
  float c0h, c0v, c1, csp;      // FP32 error-bound constants (see host code)
  float cdf;                    // per unit: |hi/lo-table pre-activation - FP64 path's|
  const double* f64;            // [K][k][2^k] row-sum tables, see struct Tabs
  const double* b64;
  const float* fd;
  const float* bd;
  const float* fh;
  const float* fl;
  const float4* fd4;            // [k][2^k] filter-interleaved, K <= 4
  const float4* fh4;
  const float4* fl4;
  // tensor-core form (Ising, L = 128, 64, 32 or 16, K <= 4, k <= 5; crbm_step_tc.cu):
  // operand images of the filter digits, null when the model has none
  const uint4* tcw;
  float tq2, tq1, tq0;          // digit scales qf 2^22, qf 2^11, qf
  float tc0h, tc0v, tc1, tcft;  // certified error constants of that form
  uint64_t seed, cid_base;
  uint32_t rk[20];              // Philox round keys (k0 + r W0, k1 + r W1), r = 0..9
  unsigned long long* step;     // device-resident step counter of the job (proposals made)
  uint32_t* bits;               // [n_chains][Wd]
  const double* T;              // [n_chains]
  double* F;                    // [n_chains]
  double* Fb;                   // [n_chains] bound on |F - F_fp64| (0: exact)
  double* Lb;                   // [n_chains] bound on |log pi - log pi_fp64| (0: exact)
  double* logpi;                // [n_chains]
  double* Ephys;                // [n_chains]
  double* obs_t;                // [n_chains][4] observables of the current lattice
  double* obs;                  // [n_chains][4] running sums
  unsigned long long* acc;      // [n_chains]
  unsigned long long* rec;      // [n_chains][2] FP64 recomputes: Bernoulli draws, MH decisions
  double* eps;                  // [n_chains][N] Kitaev: single-fermion energies of the current
                                // lattice, ascending (written by modes 1 and 2 only)
  double* trace;                // optional [trace_cap][n_chains]: E_phys after step t at row
  unsigned long long trace_base;  // t - trace_base, for 0 <= t - trace_base < trace_cap
  long long trace_cap;
};

// E_phys of chain c after step t into the job's trace, if one is set and t is inside it.
__device__ __forceinline__ void trace_store(const JobDev& jb, int c, unsigned long long t, double E) {
  if (jb.trace == nullptr) return;
  const long long r = (long long)(t - jb.trace_base);
  if (t >= jb.trace_base && r < jb.trace_cap) jb.trace[r * jb.n_chains + c] = E;
}

struct LaunchParams {
  // mode 0: S proposals; 1: evaluate the current state; 2: one uncorrected
  // proposal of the tempering RBM chains of job[0] and its exchange with the
  // physical chains of job[1] (n_jobs = 1);
  // 3: S local-update Metropolis sweeps, where correct = 1 adds each sweep's
  // observables to the sums (0: the exchange kernel that follows does)
  int n_jobs, S, g, correct, mode;
  int tile_begin[kMaxJobs + 1];
  int* err;
  // tensor-core kernel (persistent CTAs): work items 0 .. total_items - 1
  // handed out by the counter *queue (zero at launch, cleared after it);
  // every device-side wait gives up after wait_limit SM clock cycles
  int* queue;
  int total_items;
  long long wait_limit;
  JobDev job[kMaxJobs];
};

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): per round the counter words x0, x2
// are multiplied (32x32 -> 64 bit) by M0, M1; the high halves are xored with
// the other two words and the key; the key is bumped by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Same rounds with the ten round keys precomputed (rk[2r], rk[2r+1]): the
// key schedule of a launch is fixed, so the kernels read it from the launch
// parameters instead of bumping the key in every call.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
  }
  return c;
}

__device__ __forceinline__ uint32_t pick(const uint4& w, int t) {
  return t == 0 ? w.x : (t == 1 ? w.y : (t == 2 ? w.z : w.w));
}

// ------------------------------------------------------- bit-row windows
// w bits (w <= 12) of row r starting at column c (0 <= c < L), periodic in the
// column: bit b of the result is site (r, (c + b) mod L).  Supports L <= 32
// and L a multiple of 32.
__device__ __forceinline__ uint32_t row_window(const uint32_t* __restrict__ bits, int L, int r,
                                               int c, int w) {
  uint32_t x;
  if ((L & 31) == 0) {
    const int WL = L >> 5, wi = c >> 5;
    const int wn = (wi + 1 == WL) ? 0 : wi + 1;
    x = __funnelshift_r(bits[r * WL + wi], bits[r * WL + wn], c & 31);
  } else {
    const int off = r * L;
    const uint32_t row =
        __funnelshift_r(bits[off >> 5], bits[(off >> 5) + 1], off & 31) & ((1u << L) - 1u);
    uint64_t rr = row;
    for (int s = L; s < 64; s += L) rr |= (uint64_t)row << s;
    x = (uint32_t)(rr >> c);
  }
  return x & ((1u << w) - 1u);
}

__device__ __forceinline__ uint32_t site_bit(const uint32_t* bits, int n) {
  return (bits[n >> 5] >> (n & 31)) & 1u;
}

// Forward codes of unit q (sites n = 4q..4q+3): m[t][a] = a*T + (bits of
// sites (i_t + a, j_t + b), b = 0..k-1, as bit b) -- the offset of the
// row-sum table entry of kernel row a for the receptive field of hidden unit
// (i_t, j_t).  When L % 4 == 0 the 4 sites share a row and one window of
// k + 3 bits per kernel row serves all of them.  kC > 0 fixes k at compile time.
template <int kC>
__device__ __forceinline__ void fwd_codes(const uint32_t* bits, int L, int N, int k, int T, int q,
                                          uint32_t (&m)[4][kC ? kC : kMaxk]) {
  constexpr int kU = kC ? kC : kMaxk;
  const uint32_t mk = (1u << k) - 1u;
  if ((L & 3) == 0) {
    const int n0 = 4 * q, i = n0 / L, j0 = n0 - i * L;
#pragma unroll
    for (int a = 0; a < kU; ++a) {
      if (kC || a < k) {
        int r = i + a;
        if (r >= L) r -= L;
        const uint32_t win = row_window(bits, L, r, j0, k + 3);
#pragma unroll
        for (int t = 0; t < 4; ++t) m[t][a] = (uint32_t)(a * T) + ((win >> t) & mk);
      }
    }
  } else {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      int n = 4 * q + t;
      if (n >= N) n = 0;
      const int i = n / L, j = n - i * L;
#pragma unroll
      for (int a = 0; a < kU; ++a) {
        if (kC || a < k) {
          int r = i + a;
          if (r >= L) r -= L;
          m[t][a] = (uint32_t)(a * T) + row_window(bits, L, r, j, k);
        }
      }
    }
  }
}

// ------------------------------------------------ Bernoulli decisions
// FP64: h = [u < sigma(x)], u = (w + 1/2) 2^-32 exactly (App. B.1 sampling).
__device__ __forceinline__ uint32_t decide64(double x, uint32_t w) {
  const double p = 1.0 / (1.0 + exp(-x));
  const double u = ((double)w + 0.5) * 0x1p-32;
  return u < p ? 1u : 0u;
}

// Special-function-unit approximations (PTX ex2/rcp/lg2, flush-to-zero).
// Their error bounds are part of the certified margins below and are checked
// exhaustively on the device by the test-suite.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// log u of an MH draw u = (w + 1/2) 2^-32 in FP32, within 2^-20 (1 + |log u|)
// of the exact value: u = m 2^e with m in [1, 2) split off its float exactly,
// lg2 of m from the special-function unit (absolute error 2^-22 on [1, 2]),
// the float rounding of u within 2^-23 relative, the sum and the ln 2
// product within 2^-24 relative each.
__device__ __forceinline__ float log_u32(uint32_t w) {
  const uint32_t ub = __float_as_uint(((float)w + 0.5f) * 0x1p-32f);
  const float lg2u = (float)((int)(ub >> 23) - 127) + lg2_approx(__uint_as_float((ub & 0x7FFFFFu) | 0x3F800000u));
  return lg2u * 0.69314718055994531f;
}

// sigma(x) in FP32: e = 2^(-x log2 e), p = 1/(1 + e).
__device__ __forceinline__ float sigmoid32(float x) {
  return rcp_approx(1.0f + ex2_approx(x * -1.4426950408889634f));
}

// FP32 decision with a certified margin: |p32 - p64| <= c0 + c1 |x| covers the
// FP32 pre-activation error, the ex2/rcp errors, the conversion of the Philox
// word, and the FP64 path's own rounding.  Returns 0/1 when the FP64 path
// takes the same decision, 2 when the FP64 code has to decide.
// The comparison runs in units of 2^-32 (p 2^32 against the Philox word), so
// c0 and c1 arrive pre-scaled by 2^32.
__device__ __forceinline__ uint32_t decide32(float x, uint32_t w, float c0, float c1) {
  const float d = fmaf(sigmoid32(x), 0x1p32f, -__uint2float_rn(w));
  const float delta = fmaf(c1, fabsf(x), c0);
  return fabsf(d) > delta ? (d > 0.0f ? 1u : 0u) : 2u;
}

// The same decision as decide32, returned as the FP32 bit and a flag that is
// 1 when the margin does not separate it (then the FP64 path decides).
__device__ __forceinline__ void decide32_split(float x, uint32_t w, float c0, float c1, uint32_t& bit,
                                               uint32_t& amb) {
  const float d = fmaf(sigmoid32(x), 0x1p32f, -__uint2float_rn(w));
  const float delta = fmaf(c1, fabsf(x), c0);
  bit = d > 0.0f ? 1u : 0u;
  amb = fabsf(d) > delta ? 0u : 1u;
}

// log(1 + e^x) without overflow.
__device__ __forceinline__ double softplus64(double x) {
  return fmax(x, 0.0) + log1p(exp(-fabs(x)));
}
// FP32: max(x, 0) + ln 2 * log2(1 + 2^(-|x| log2 e)).
__device__ __forceinline__ float softplus32(float x) {
  const float e = ex2_approx(fabsf(x) * -1.4426950408889634f);
  return fmaxf(x, 0.0f) + 0.69314718055994531f * lg2_approx(1.0f + e);
}

// Store the 4-bit result of unit q: 8 consecutive lanes own the 8 units of
// one word and OR their nibbles together.  Every lane of the warp must call.
__device__ __forceinline__ void store_nibble(uint32_t* plane, int q, uint32_t nib, bool act) {
  uint32_t x = act ? (nib << (4 * (q & 7))) : 0u;
  x |= __shfl_xor_sync(kFull, x, 1);
  x |= __shfl_xor_sync(kFull, x, 2);
  x |= __shfl_xor_sync(kFull, x, 4);
  if (act && (q & 7) == 0) plane[q >> 3] = x;
}

// One chain's thread group: tpc threads (a power of two >= 8), rank r.
struct Grp {
  int c;          // chain index within the job
  int gl;         // group index within the CTA
  int r, tpc;
  bool active;    // c < n_chains
  uint32_t cid;   // chain id (Philox counter word 3)
};

// Deterministic sum of NV doubles over a chain's group; the result is valid in
// the leader (r == 0).  Every thread of the CTA must call (it may sync).
template <int NV>
__device__ __forceinline__ void grp_reduce(double (&x)[NV], const Grp& g, double* scratch) {
  const int span = g.tpc < 32 ? g.tpc : 32;
  for (int o = 1; o < span; o <<= 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] += __shfl_xor_sync(kFull, x[v], o);
  }
  if (g.tpc > 32) {
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) scratch[warp * NV + v] = x[v];
    }
    __syncthreads();
    if (g.r == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double s = 0.0;
        for (int w = 0; w < g.tpc / 32; ++w) s += scratch[(warp + w) * NV + v];
        x[v] = s;
      }
    }
    __syncthreads();
  }
}

// grp_reduce for a warp-aligned group with scratch of its own (NV * tpc / 32
// doubles), synchronising only the group: the same order of additions, the
// result valid in the leader (r == 0).
template <int NV, bool MULTI>
__device__ __forceinline__ void grp_reduce_local(double (&x)[NV], const Grp& g, double* scratch);

// Barrier of one chain's thread group (warp-aligned groups of 32 .. blockDim
// threads): the CTA barrier when the group is the whole CTA, the warp's when it
// is one warp, else a named barrier of its own (id 1 + group index; a CTA holds
// at most 8 groups).  Only the group's threads take part, so groups may run
// different branches between two of their barriers.  MULTI = false: the
// caller's CTAs hold one group each, and this is the CTA barrier (code without
// named barriers, which would reserve all of the CTA's barrier slots).
template <bool MULTI>
__device__ __forceinline__ void grp_sync(const Grp& g) {
  if (!MULTI || g.tpc == (int)blockDim.x) {
    __syncthreads();
  } else if (g.tpc == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;\n" :: "r"(1 + g.gl), "r"(g.tpc) : "memory");
  }
}

// Deterministic sum over a chain's (warp-aligned) group, returned to every
// thread of it: a butterfly within each warp, then the warps' partials added
// in warp order -- the order of block_sum for a CTA of tpc threads, so a group
// gives the same bits as a CTA of its size.  scratch: 32 doubles of the group.
template <bool MULTI>
__device__ __forceinline__ double grp_sum(double x, const Grp& g, double* scratch) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) x += __shfl_xor_sync(kFull, x, o);
  const int r = MULTI ? g.r : (int)threadIdx.x, tpc = MULTI ? g.tpc : (int)blockDim.x;
  const int warp = r >> 5, nw = tpc >> 5;
  grp_sync<MULTI>(g);
  if ((r & 31) == 0) scratch[warp] = x;
  grp_sync<MULTI>(g);
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += scratch[w];
  grp_sync<MULTI>(g);
  return s;
}

template <int NV, bool MULTI>
__device__ __forceinline__ void grp_reduce_local(double (&x)[NV], const Grp& g, double* scratch) {
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] += __shfl_xor_sync(kFull, x[v], o);
  }
  if (g.tpc > 32) {
    const int warp = g.r >> 5;
    if ((g.r & 31) == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) scratch[warp * NV + v] = x[v];
    }
    grp_sync<MULTI>(g);
    if (g.r == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double s = 0.0;
        for (int w = 0; w < g.tpc / 32; ++w) s += scratch[w * NV + v];
        x[v] = s;
      }
    }
    grp_sync<MULTI>(g);
  }
}

// Deterministic block-wide sum, result returned to every thread.
__device__ __forceinline__ double block_sum(double x, double* scratch) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) x += __shfl_xor_sync(kFull, x, o);
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) scratch[warp] = x;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += scratch[w];
  __syncthreads();
  return s;
}

// Row-sum tables of one model (index (f*k + a)*T + code, T = 2^k):
//   f64/b64   FP64, forward code / raw backward window (FP64 path; global
//             copies of them serve the mixed path's FP64 recomputes)
//   fd/bd     FP32 roundings of f64/b64 (mixed-path decisions)
//   fh/fl     hi/lo split of f64 (mixed-path free energy)
//   fd4/fh4/fl4  the same forward tables with the filter index innermost,
//             in shared memory replicated 8 times, entry e of copy c at
//             float4 index 8 e + c; thread t reads copy t % 8 (the pointer
//             below already includes + t % 8, so entry e is at [e << 3]):
//             the 8 threads of a quarter-warp hit 8 distinct bank groups
//             whatever their codes, so a 16-byte table load never conflicts;
//             (a*T + code)*4 + f, for K <= 4 (zero-padded): one 16-byte load
//             serves all filters of a site
struct Tabs {
  const double* f64;
  const double* b64;
  const float* fd;
  const float* bd;
  const float* fh;
  const float* fl;
  const float4* fd4;
  const float4* fh4;
  const float4* fl4;
  int T;
};

__device__ __forceinline__ float comp(const float4& v, int f) {
  return f == 0 ? v.x : (f == 1 ? v.y : (f == 2 ? v.z : v.w));
}

// FP64 recomputes of the mixed path (rare; kept out of line so that the FP32
// fast path keeps its registers).  Same tables (global copies), same order.
static __device__ __noinline__ uint32_t recompute_hidden(const JobDev& jb, int f, const uint32_t* m, int k,
                                                         int T, uint32_t w) {
  double x = jb.hb[f];
  const int base = f * k * T;
  for (int a = 0; a < k; ++a) x += __ldg(jb.f64 + base + m[a]);
  return decide64(x, w);
}

__device__ __forceinline__ int bwd_row(int i, int a, int L) {
  int r = i - a;
  return r < 0 ? r + L : r;
}

// This site's visible pre-activation with the FP64 tables, in the FP64 path's order.
static __device__ __noinline__ uint32_t recompute_visible(const JobDev& jb, const uint32_t* h, int P, int n,
                                                          uint32_t w) {
  const int L = jb.L, K = jb.K, k = jb.k, T = 1 << k;
  const int i = n / L, j = n - i * L;
  int c = j - (k - 1);
  if (c < 0) c += L;
  double x = jb.vb;
  for (int a = 0; a < k; ++a) {
    const int r = bwd_row(i, a, L);
    for (int f = 0; f < K; ++f) x += __ldg(jb.b64 + (f * k + a) * T + row_window(h + f * P, L, r, c, k));
  }
  return decide64(x, w);
}

// ------------------------------------------------- LCRBM (open columns)
// Column class of hidden column j: left edge columns 0..e-1, right edge
// columns e..2e-1, bulk 2e (Sec. IV, open boundary conditions).
__device__ __forceinline__ int lc_class(int j, int L, int e) {
  return j < e ? j : (j >= L - e ? e + (j - (L - e)) : 2 * e);
}

// FP64 pre-activation of filter f of an LCRBM at site n from the forward
// codes m (computed with wrap): the window is cut at the open column edge
// (bits b >= L - j dropped) and the table of the column's class is used.
template <int kU>
__device__ __forceinline__ double lc_preact64(const JobDev& jb, const double* f64, int f, const uint32_t (&m)[kU],
                                              int n, int k, int T) {
  const int L = jb.L, j = n % L;
  const int base = (lc_class(j, L, jb.lc_edge) * jb.K + f) * k * T;
  const uint32_t keep = (j + k > L) ? ((1u << (L - j)) - 1u) : 0xFFFFFFFFu;
  double x = jb.hb[f];
#pragma unroll
  for (int a = 0; a < kU; ++a) {
    if (a < k) {
      const uint32_t code = (m[a] - (uint32_t)(a * T)) & keep;
      x += f64[base + a * T + (int)code];
    }
  }
  return x;
}

// FP64 visible pre-activation of an LCRBM at site n: v_bias plus, for every
// hidden unit (f, i-a, j-b) with j - b >= 0, its class kernel's weight
// W[c(j-b)][f][a][b] (the table entry of the single-bit code 1 << b) if set.
__device__ inline double lc_visible64(const JobDev& jb, const double* f64, const uint32_t* h, int P, int n,
                                      int k, int T) {
  const int L = jb.L, i = n / L, j = n - i * L;
  double x = jb.vb;
  for (int a = 0; a < k; ++a) {
    const int r = (i - a < 0) ? i - a + L : i - a;
    for (int f = 0; f < jb.K; ++f) {
      const uint32_t* pl = h + f * P;
      for (int b = 0; b < k && b <= j; ++b) {
        const int jc = j - b;
        if (site_bit(pl, r * L + jc))
          x += f64[((lc_class(jc, L, jb.lc_edge) * jb.K + f) * k + a) * T + (1 << b)];
      }
    }
  }
  return x;
}

// ------------------------------------------------- hidden half-step
// h^f_ij = [u < sigma(h_bias^f + sum_ab W^f_ab v_(i+a)(j+b))]  (Eq. B2, Eq. 12)
// FP64 order (shared with the mixed path's recompute): h_bias, then kernel
// rows a = 0..k-1.  KC, kC > 0 fix K and k at compile time (0: runtime).
template <int PREC, int KC, int kC>
__device__ void hidden_phase(const JobDev& jb, const Tabs& tb, const Grp& g, const uint32_t* v,
                             uint32_t* h, int P, uint32_t step, int sub, unsigned& nrec) {
  constexpr int kU = kC ? kC : kMaxk;
  const int L = jb.L, N = jb.N, K = KC ? KC : jb.K, k = kC ? kC : jb.k, T = tb.T;
  const int nblk = (N + 3) >> 2;
  const int iters = (nblk + g.tpc - 1) / g.tpc;
  const uint32_t k0 = (uint32_t)jb.seed, k1 = (uint32_t)(jb.seed >> 32);
  for (int it = 0; it < iters; ++it) {
    const int q = g.r + it * g.tpc;
    const bool act = g.active && q < nblk;
    uint32_t m[4][kU];
    fwd_codes<kC>(v, L, N, k, T, act ? q : 0, m);
    if (PREC == kMixed && KC == 4) {
      // all four filters per site from the filter-interleaved table
      uint4 w[4];
#pragma unroll
      for (int f = 0; f < 4; ++f)
        w[f] = philox4x32_10_rk(make_uint4((uint32_t)q, (uint32_t)(sub * 5 + f), step, g.cid), jb.rk);
      uint32_t nib[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float4 x = make_float4(jb.hb32[0], jb.hb32[1], jb.hb32[2], jb.hb32[3]);
#pragma unroll
        for (int a = 0; a < kU; ++a) {
          if (kC || a < k) {
            const float4 e = tb.fd4[m[t][a] << 3];
            x.x += e.x;
            x.y += e.y;
            x.z += e.z;
            x.w += e.w;
          }
        }
        const bool site = act && 4 * q + t < N;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          uint32_t bit = decide32(comp(x, f), pick(w[f], t), jb.c0h, jb.c1);
          if (bit == 2u) {
            uint32_t mm[kMaxk];
#pragma unroll
            for (int a = 0; a < kU; ++a) mm[a] = m[t][a];
            bit = recompute_hidden(jb, f, mm, k, T, pick(w[f], t));
            if (site) ++nrec;
          }
          if (site) nib[f] |= bit << t;
        }
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) store_nibble(h + f * P, q, nib[f], act);
      continue;
    }
    for (int f = 0; f < K; ++f) {
      const uint4 w = philox4x32_10_rk(make_uint4((uint32_t)q, (uint32_t)(sub * (K + 1) + f), step, g.cid), jb.rk);
      const int base = f * k * T;
      uint32_t nib = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        uint32_t bit;
        if (PREC == kFP64) {
          double x = jb.hb[f];
          if (KC == 0 && jb.lc_edge) {
            x = lc_preact64<kU>(jb, tb.f64, f, m[t], (act && 4 * q + t < N) ? 4 * q + t : 0, k, T);
          } else {
#pragma unroll
            for (int a = 0; a < kU; ++a) if (kC || a < k) x += tb.f64[base + m[t][a]];
          }
          bit = decide64(x, pick(w, t));
        } else {
          float x = jb.hb32[f];
#pragma unroll
          for (int a = 0; a < kU; ++a) if (kC || a < k) x += tb.fd[base + m[t][a]];
          bit = decide32(x, pick(w, t), jb.c0h, jb.c1);
          if (bit == 2u) {
            uint32_t mm[kMaxk];
#pragma unroll
            for (int a = 0; a < kU; ++a) mm[a] = m[t][a];
            bit = recompute_hidden(jb, f, mm, k, T, pick(w, t));
            if (act && 4 * q + t < N) ++nrec;
          }
        }
        if (act && 4 * q + t < N) nib |= bit << t;
      }
      store_nibble(h + f * P, q, nib, act);
    }
  }
}

// ------------------------------------------------- visible half-step
// v'_ij = [u < sigma(v_bias + sum_f sum_ab W^f_ab h^f_(i-a)(j-b))]  (Eq. B3)
// The window of hidden row i - a starting at column j - (k-1) holds, as bit
// k-1-b, the unit h_(i-a)(j-b); the backward tables are indexed by that raw
// window.  Order: v_bias, then kernel rows a, then filters f.
template <int PREC, int KC, int kC>
__device__ void visible_phase(const JobDev& jb, const Tabs& tb, const Grp& g, const uint32_t* h,
                              uint32_t* vp, int P, uint32_t step, int sub, unsigned& nrec) {
  constexpr int kU = kC ? kC : kMaxk;
  constexpr int KU = KC ? KC : kMaxK;
  const int L = jb.L, N = jb.N, K = KC ? KC : jb.K, k = kC ? kC : jb.k, T = tb.T;
  const uint32_t mk = (1u << k) - 1u;
  const int nblk = (N + 3) >> 2;
  const int iters = (nblk + g.tpc - 1) / g.tpc;
  const uint32_t k0 = (uint32_t)jb.seed, k1 = (uint32_t)(jb.seed >> 32);
  const bool rows4 = (L & 3) == 0;
  for (int it = 0; it < iters; ++it) {
    const int q = g.r + it * g.tpc;
    const bool act = g.active && q < nblk;
    const int qq = act ? q : 0;
    double x64[4];
    float x32[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      x64[t] = jb.vb;
      x32[t] = jb.vb32;
    }
    if (rows4) {
      const int n0 = 4 * qq, i = n0 / L, j0 = n0 - i * L;
      int c = j0 - (k - 1);
      if (c < 0) c += L;
#pragma unroll
      for (int a = 0; a < kU; ++a) {
        if (kC || a < k) {
          const int r = bwd_row(i, a, L);
          // word offsets of this window, shared by the K hidden planes
          int o0, o1, sh;
          const bool wide = (L & 31) == 0;
          if (wide) {
            const int WL = L >> 5, wi = c >> 5;
            o0 = r * WL + wi;
            o1 = r * WL + ((wi + 1 == WL) ? 0 : wi + 1);
            sh = c & 31;
          } else {
            const int off = r * L;
            o0 = off >> 5;
            o1 = o0 + 1;
            sh = off & 31;
          }
#pragma unroll
          for (int f = 0; f < KU; ++f) {
            if (KC || f < K) {
              const uint32_t* pl = h + f * P;
              uint32_t win;
              if (wide) {
                win = __funnelshift_r(pl[o0], pl[o1], sh);
              } else {
                const uint32_t row = __funnelshift_r(pl[o0], pl[o1], sh) & ((1u << L) - 1u);
                uint64_t rr = row;
                for (int s2 = L; s2 < 64; s2 += L) rr |= (uint64_t)row << s2;
                win = (uint32_t)(rr >> c);
              }
              const int base = (f * k + a) * T;
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                const uint32_t code = (win >> t) & mk;
                if (PREC == kFP64) x64[t] += tb.b64[base + code];
                else x32[t] += tb.bd[base + code];
              }
            }
          }
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        int n = 4 * qq + t;
        if (n >= N) n = 0;
        const int i = n / L, j = n - i * L;
        int c = j - (k - 1);
        if (c < 0) c += L;
        for (int a = 0; a < k; ++a) {
          const int r = bwd_row(i, a, L);
          for (int f = 0; f < K; ++f) {
            const uint32_t code = row_window(h + f * P, L, r, c, k);
            const int base = (f * k + a) * T;
            if (PREC == kFP64) x64[t] += tb.b64[base + code];
            else x32[t] += tb.bd[base + code];
          }
        }
      }
    }
    if (PREC == kFP64 && KC == 0 && jb.lc_edge) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int n = 4 * qq + t;
        x64[t] = lc_visible64(jb, tb.f64, h, P, n < N ? n : 0, k, T);
      }
    }
    const uint4 w = philox4x32_10_rk(make_uint4((uint32_t)q, (uint32_t)(sub * (K + 1) + K), step, g.cid), jb.rk);
    uint32_t nib = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (act && 4 * q + t < N) {
        uint32_t bit;
        if (PREC == kFP64) {
          bit = decide64(x64[t], pick(w, t));
        } else {
          bit = decide32(x32[t], pick(w, t), jb.c0v, jb.c1);
          if (bit == 2u) {
            bit = recompute_visible(jb, h, P, 4 * q + t, pick(w, t));
            ++nrec;
          }
        }
        nib |= bit << t;
      }
    }
    store_nibble(vp, q, nib, act);
  }
}

// ------------------------------------------------- free energy + lattice sums
// F(v) = -v_bias sum v - sum_{f,i,j} softplus(h_bias^f + (W^f * v)_ij)   (Eq. 13)
// Per-thread partial sums: out[0] = sum softplus (FP64 order, or FP32 with
// Kahan compensation), out[1] = data part of the FP32 error bound (mixed),
// out[2] = number of ones, out[3] = number of unequal nearest-neighbour pairs
// (Ising) or of hexagons with flux -1 (Kitaev).
template <int PREC, int KC, int kC>
__device__ void free_phase(const JobDev& jb, const Tabs& tb, const Grp& g, const uint32_t* v,
                           double (&out)[4]) {
  constexpr int kU = kC ? kC : kMaxk;
  const int L = jb.L, N = jb.N, K = KC ? KC : jb.K, k = kC ? kC : jb.k, T = tb.T;
  const int nblk = (N + 3) >> 2;
  const int iters = (nblk + g.tpc - 1) / g.tpc;
  double s64 = 0.0;
  float s32 = 0.0f, c32 = 0.0f, sabs = 0.0f, ssp = 0.0f;
  int ones = 0, pairs = 0;
  for (int it = 0; it < iters; ++it) {
    const int q = g.r + it * g.tpc;
    const bool act = g.active && q < nblk;
    if (!act) continue;
    uint32_t m[4][kU];
    fwd_codes<kC>(v, L, N, k, T, q, m);
    if (PREC == kMixed && KC == 4) {
      float sp[4][4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float4 xh = make_float4(jb.hb_hi[0], jb.hb_hi[1], jb.hb_hi[2], jb.hb_hi[3]);
        float4 xl = make_float4(jb.hb_lo[0], jb.hb_lo[1], jb.hb_lo[2], jb.hb_lo[3]);
#pragma unroll
        for (int a = 0; a < kU; ++a) {
          if (kC || a < k) {
            const float4 eh = tb.fh4[m[t][a] << 3], el = tb.fl4[m[t][a] << 3];
            xh.x += eh.x; xh.y += eh.y; xh.z += eh.z; xh.w += eh.w;
            xl.x += el.x; xl.y += el.y; xl.z += el.z; xl.w += el.w;
          }
        }
        const bool site = 4 * q + t < N;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const float x = comp(xh, f) + comp(xl, f);
          sp[t][f] = site ? softplus32(x) : 0.0f;
          sabs += site ? fabsf(x) : 0.0f;
        }
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const float us = (sp[0][f] + sp[1][f]) + (sp[2][f] + sp[3][f]);
        ssp += us;
        const float y = us - c32;          // Kahan summation of the unit sums
        const float tt = s32 + y;
        c32 = (tt - s32) - y;
        s32 = tt;
      }
    } else {
      for (int f = 0; f < K; ++f) {
        const int base = f * k * T;
        if (PREC == kFP64) {
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            if (4 * q + t < N) {
              double x = jb.hb[f];
              if (KC == 0 && jb.lc_edge) {
                x = lc_preact64<kU>(jb, tb.f64, f, m[t], 4 * q + t, k, T);
              } else {
#pragma unroll
                for (int a = 0; a < kU; ++a) if (kC || a < k) x += tb.f64[base + m[t][a]];
              }
              s64 += softplus64(x);
            }
          }
        } else {
          float sp[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            sp[t] = 0.0f;
            if (4 * q + t < N) {
              float xh = jb.hb_hi[f], xl = jb.hb_lo[f];
#pragma unroll
              for (int a = 0; a < kU; ++a) {
                if (kC || a < k) {
                  xh += tb.fh[base + m[t][a]];
                  xl += tb.fl[base + m[t][a]];
                }
              }
              const float x = xh + xl;
              sp[t] = softplus32(x);
              sabs += fabsf(x);
            }
          }
          const float us = (sp[0] + sp[1]) + (sp[2] + sp[3]);
          ssp += us;
          const float y = us - c32;
          const float tt = s32 + y;
          c32 = (tt - s32) - y;
          s32 = tt;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int n = 4 * q + t;
      if (n < N) {
        const int i = n / L, j = n - i * L;
        const uint32_t b0 = m[t][0] & 1u;
        ones += (int)b0;
        if (jb.kind == kIsing) {
          const uint32_t right = (k >= 2) ? ((m[t][0] >> 1) & 1u) : site_bit(v, i * L + (j + 1 == L ? 0 : j + 1));
          const uint32_t down = (k >= 2) ? ((m[t][kU > 1 ? 1 : 0] - (uint32_t)T) & 1u)
                                         : site_bit(v, (i + 1 == L ? 0 : i + 1) * L + j);
          pairs += (int)(b0 ^ right) + (int)(b0 ^ down);
        } else {
          // the hexagon of cell r holds the z-bonds r and r - e1 + e2 (with
          // open columns the hexagons of column L-1 do not exist)
          const int i2 = (i == 0) ? L - 1 : i - 1, j2 = (j + 1 == L) ? 0 : j + 1;
          if (!(jb.lc_edge && j + 1 == L)) pairs += (int)(b0 ^ site_bit(v, i2 * L + j2));
        }
      }
    }
  }
  if (PREC == kFP64) {
    out[0] = s64;
    out[1] = 0.0;
  } else {
    out[0] = (double)s32;
    // x rounding + ex2 argument: 2^-23 |x|; pairwise, Kahan and final add: 6 2^-24 sp;
    // 1.001 covers the FP32 accumulation of these two sums themselves
    out[1] = ((double)sabs * 0x1p-23 + (double)ssp * (6.0 * 0x1p-24)) * 1.001;
  }
  out[2] = (double)ones;
  out[3] = (double)pairs;
}

// --------------------------------------------------- Kitaev log-weight
// FP64 eigen-stage for one lattice by the whole CTA.  A = M^T M (Sec. IV,
// M_bw = 2 J_a u_bw) is reduced to tridiagonal form by Householder
// reflections, its eigenvalues mu_l = eps_l^2 are found by bisection with
// Sturm counts, and log pi = sum_l log 2cosh(beta eps_l / 2).
// Packed lower triangle of a symmetric N x N matrix: element (i, c), c <= i.
__device__ __forceinline__ int tri(int i, int c) { return i * (i + 1) / 2 + c; }
// Lanes per row of a group's matrix-vector product over m rows with nt
// threads: the largest power of two H <= 32 with H m <= nt (at least 1).
__device__ __forceinline__ int row_split(int m, int nt) {
  int H = 1;
  while (H < 32 && 2 * H * m <= nt) H <<= 1;
  return H;
}

// Thread tid of nt visiting a packed triangle of R rows (row r: columns
// 0..r) with stride nt: rows p and R-1-p side by side form folded row p,
// R+1 long, so the thread's next element is a fixed step away in the folded
// rows (for odd R the middle row is the last folded row's first half).
// Every element is visited once, neighbouring threads take neighbouring
// elements, and no walk across the short rows is needed.
struct FoldWalk {
  int R, p, o, dp, dq;
  __device__ __forceinline__ FoldWalk(int rows, int tid, int nt) : R(rows) {
    p = tid / (rows + 1);
    o = tid - p * (rows + 1);
    dp = nt / (rows + 1);
    dq = nt - dp * (rows + 1);
  }
  __device__ __forceinline__ void rc(int& r, int& c) const {
    const bool first = o <= p;
    r = first ? p : R - 1 - p;
    c = first ? o : o - p - 1;
  }
  __device__ __forceinline__ void next() {
    o += dq;
    p += dp;
    if (o > R) {
      o -= R + 1;
      ++p;
    }
  }
};

struct KitaevWork {
  double* A;       // packed lower triangle, N (N+1) / 2 entries
  double* d;       // N
  double* e;       // N
  double* vv;      // N
  double* pw;      // N
  double* sc;      // 64 doubles
  float* d32;      // N   FP32 copies of the tridiagonal for eigenvalue isolation
  float* e32;      // N   (squared off-diagonals)
};

// Number of eigenvalues below x of the symmetric tridiagonal (d, off-diagonal^2
// = e2): sign changes of p_{-1} = 1, p_0, ..., p_{N-1} with
// p_i = (d_i - x) p_{i-1} - e2_{i-1} p_{i-2} (Sturm).  A zero p_i takes the sign
// opposite to p_{i-1}.  The pair (p_i, p_{i-1}) is rescaled by 2^-+500 when
// it leaves [2^-500, 2^500].  Signs and exponents are read from the bit
// patterns with integer operations: only the recurrence itself uses the FP64
// pipe (three operations per step).
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int N, double x) {
  double pp = 1.0, p = d[0] - x;
  int hi = __double2hiint(p);
  uint32_t sprev = 0u;                                           // sign of p_{-1} = +1
  uint32_t s = ((hi & 0x7fffffff) | __double2loint(p)) == 0 ? 1u : ((uint32_t)hi >> 31);
  int cnt = (int)(s ^ sprev);
  sprev = s;
  for (int i = 1; i < N; ++i) {
    const double pn = fma(-e2[i - 1], pp, (d[i] - x) * p);
    pp = p;
    p = pn;
    hi = __double2hiint(p);
    const uint32_t zero = ((hi & 0x7fffffff) | __double2loint(p)) == 0;
    s = zero ? (sprev ^ 1u) : ((uint32_t)hi >> 31);
    cnt += (int)(s ^ sprev);
    sprev = s;
    const int ex = (hi >> 20) & 0x7ff;                           // biased exponent of p
    if (ex > 1023 + 500) {
      p *= 0x1p-500;
      pp *= 0x1p-500;
    } else if (ex < 1023 - 500 && ((__double2hiint(pp) >> 20) & 0x7ff) < 1023 - 500) {
      p *= 0x1p+500;
      pp *= 0x1p+500;
    }
  }
  return cnt;
}

// FP32 Sturm count (same recurrence, rescaled by 2^-+60): used only to
// isolate eigenvalues; every bracket it yields is checked with FP64 counts.
__device__ __forceinline__ int sturm_count32(const float* d, const float* e2, int N, float x) {
  float pp = 1.0f, p = d[0] - x;
  uint32_t b = __float_as_uint(p);
  uint32_t sprev = 0u;
  uint32_t s = (b << 1) == 0u ? 1u : (b >> 31);
  int cnt = (int)(s ^ sprev);
  sprev = s;
  for (int i = 1; i < N; ++i) {
    const float pn = fmaf(-e2[i - 1], pp, (d[i] - x) * p);
    pp = p;
    p = pn;
    b = __float_as_uint(p);
    s = (b << 1) == 0u ? (sprev ^ 1u) : (b >> 31);
    cnt += (int)(s ^ sprev);
    sprev = s;
    const int ex = (int)((b >> 23) & 0xffu);
    if (ex > 127 + 60) {
      p *= 0x1p-60f;
      pp *= 0x1p-60f;
    } else if (ex < 127 - 60 && (int)((__float_as_uint(pp) >> 23) & 0xffu) < 127 - 60) {
      p *= 0x1p+60f;
      pp *= 0x1p+60f;
    }
  }
  return cnt;
}

// Shared start of the eigenvalues' FP32 bisections: G points strictly inside
// the (FP32) Gershgorin interval, point k at lo + (k + 1) h with
// h = (hi - lo) / (G + 1), and the FP32 Sturm count at each, one point per
// thread of the group.  The count at a point is the number of eigenvalues
// below it, so eigenvalue idx lies between the last point whose count is
// <= idx and the next one: about log2(G + 1) rounds of bisection that every
// eigenvalue would otherwise repeat on its own are taken in one round.  The
// counts live in the reduced matrix's storage, free by then beyond the
// first 2N doubles (at most N^2 - 3N ints).
struct EigGrid {
  const int* cnt;
  int G;
  float lo, hi, h;
  __device__ __forceinline__ float x(int k) const { return __fmaf_rn((float)(k + 1), h, lo); }
  // [lo32, hi32]: neighbouring grid points (or interval ends) with
  // count(lo32) <= idx < count(hi32) as computed; the bisection goes on from
  // there, and the verification after it falls back to the Gershgorin interval
  // should the FP32 counts not be monotone
  __device__ __forceinline__ void bracket(int idx, float& lo32, float& hi32) const {
    int a = 0, b = G;
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (cnt[mid] > idx) b = mid; else a = mid + 1;
    }
    lo32 = a == 0 ? lo : x(a - 1);
    hi32 = a == G ? hi : x(a);
  }
};

// Fill the grid (every thread of the group calls; the caller syncs the group
// before the counts are read).  d32 / e32 and the interval must be final.
__device__ __forceinline__ EigGrid eig_grid(const KitaevWork& wk, int N, double glo, double ghi, int tid, int nt) {
  EigGrid gr;
  int* cnt = reinterpret_cast<int*>(wk.A + 2 * N);
  gr.cnt = cnt;
  gr.G = min(nt, N * N - 3 * N);
  gr.lo = (float)glo;
  gr.hi = (float)ghi;
  gr.h = (gr.hi - gr.lo) / (float)(gr.G + 1);
  if (tid < gr.G) cnt[tid] = sturm_count32(wk.d32, wk.e32, N, gr.x(tid));
  return gr;
}

// FP64 Sturm count together with p_N(x) and p_N'(x) (for a Newton step):
// p_i' = (d_i - x) p_{i-1}' - p_{i-1} - e2_{i-1} p_{i-2}', all four values of a
// step rescaled together.  Five FP64 operations per step.
struct SturmNewton {
  int cnt;
  double p, dp;
};

__device__ __forceinline__ SturmNewton sturm_newton(const double* d, const double* e2, int N, double x) {
  double pp = 1.0, p = d[0] - x, dpp = 0.0, dp = -1.0;
  int hi = __double2hiint(p);
  uint32_t sprev = 0u;
  uint32_t s = ((hi & 0x7fffffff) | __double2loint(p)) == 0 ? 1u : ((uint32_t)hi >> 31);
  int cnt = (int)(s ^ sprev);
  sprev = s;
  for (int i = 1; i < N; ++i) {
    const double dx = d[i] - x;
    const double pn = fma(-e2[i - 1], pp, dx * p);
    const double dpn = fma(-e2[i - 1], dpp, fma(dx, dp, -p));
    pp = p;
    p = pn;
    dpp = dp;
    dp = dpn;
    hi = __double2hiint(p);
    const uint32_t zero = ((hi & 0x7fffffff) | __double2loint(p)) == 0;
    s = zero ? (sprev ^ 1u) : ((uint32_t)hi >> 31);
    cnt += (int)(s ^ sprev);
    sprev = s;
    const int ex = max((hi >> 20) & 0x7ff, (__double2hiint(dp) >> 20) & 0x7ff);
    if (ex > 1023 + 500) {
      p *= 0x1p-500;
      pp *= 0x1p-500;
      dp *= 0x1p-500;
      dpp *= 0x1p-500;
    } else if (ex < 1023 - 500 && max((__double2hiint(pp) >> 20) & 0x7ff, (__double2hiint(dpp) >> 20) & 0x7ff) <
                                      1023 - 500) {
      p *= 0x1p+500;
      pp *= 0x1p+500;
      dp *= 0x1p+500;
      dpp *= 0x1p+500;
    }
  }
  return {cnt, p, dp};
}

// Eigenvalue idx (ascending) of the tridiagonal: FP32 bisection isolates it,
// two FP64 Sturm counts verify the bracket (falling back to the Gershgorin
// interval), then safeguarded Newton steps on p_N refine it in FP64; every
// iterate updates the bracket through its Sturm count, and a step that leaves
// the bracket is replaced by bisection.
__device__ __forceinline__ double eigen_idx(const KitaevWork& wk, const EigGrid& gr, int N, int idx, double glo,
                                           double ghi) {
  const double range = fmax(ghi - glo, 1e-300);
  float lo32, hi32;
  gr.bracket(idx, lo32, hi32);
  const float w32 = (float)(range * 0x1p-20);
  for (int it = 0; it < 48 && hi32 - lo32 > w32; ++it) {
    const float mid = 0.5f * (lo32 + hi32);
    if (!(mid > lo32 && mid < hi32)) break;
    if (sturm_count32(wk.d32, wk.e32, N, mid) > idx) hi32 = mid; else lo32 = mid;
  }
  const double pad = 0x1p-14 * range;
  double lo = fmax(glo, (double)lo32 - pad), hi = fmin(ghi, (double)hi32 + pad);
  if (sturm_count(wk.d, wk.vv, N, lo) > idx) lo = glo;
  if (sturm_count(wk.d, wk.vv, N, hi) <= idx) hi = ghi;
  const double tol_abs = 1e-15 * range;
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 100; ++it) {
    const double tol = fmax(tol_abs, 4.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi)));
    if (hi - lo <= tol) {
      x = 0.5 * (lo + hi);
      break;
    }
    const SturmNewton r = sturm_newton(wk.d, wk.vv, N, x);
    if (r.cnt > idx) hi = x; else lo = x;
    const double step = r.p / r.dp;
    double xn = x - step;
    // a Newton step below the tolerance that stays in the bracket has found
    // the root: stop before the bracket test below can turn it into bisection
    // (x may sit on the root itself, which then is one end of the bracket)
    if (fabs(step) <= tol && xn >= lo && xn <= hi) {
      x = xn;
      break;
    }
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (fabs(xn - x) <= tol) {
      x = xn;
      break;
    }
    x = xn;
  }
  return x;
}

// One single-fermion level's share of log pi, e and c_f (Sec. IV):
// log 2cosh x, -(eps/2) tanh x and x^2 sech^2 x with x = beta eps / 2.
__device__ __forceinline__ void thermal_add(double eps, double beta, double& lp, double& en, double& cf) {
  const double x = 0.5 * beta * eps;
  const double qx = exp(-2.0 * x);
  lp += x + log1p(qx);
  en += -0.5 * eps * (1.0 - qx) / (1.0 + qx);
  cf += x * x * 4.0 * qx / ((1.0 + qx) * (1.0 + qx));
}

// eps_out (optional, device memory): the N energies eps, ascending.
// open_cols: the lattice is open along j (the y-bonds from column L-1 to
// column 0 are absent), the physics of the LCRBM's open boundary conditions.
// Run by the chain's thread group g (warp-aligned) with its own work areas wk;
// every thread of the group calls, and only the group synchronises (MULTI:
// see grp_sync).
template <bool MULTI>
__device__ inline void kitaev_logpi64(const Grp& g, const uint32_t* v, int L, const double* J, double beta,
                               const KitaevWork& wk, double (&res)[3], double* eps_out = nullptr,
                               bool open_cols = false) {
  const int N = L * L, tid = MULTI ? g.r : (int)threadIdx.x, nt = MULTI ? g.tpc : (int)blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double* A = wk.A;
  const double tx = 2.0 * J[0], ty = 2.0 * J[1], tz = 2.0 * J[2];
  // A = M^T M, row w accumulated in a fixed order (z, x, y bond of w, then the
  // three whites of that black site)
  for (int w = tid; w < N; w += nt) {
    double* row = A + tri(w, 0);                    // lower-triangle row w: columns 0..w
    for (int c = 0; c <= w; ++c) row[c] = 0.0;
    const int i = w / L, j = w - i * L;
    for (int typ = 0; typ < 3; ++typ) {
      int bi = i, bj = j;
      if (typ == 1) bi = (i == 0) ? L - 1 : i - 1;
      if (typ == 2) bj = (j == 0) ? L - 1 : j - 1;
      if (typ == 2 && open_cols && j == 0) continue;      // this y-bond crosses the open cut
      const int b = bi * L + bj;
      const double mz = site_bit(v, b) ? tz : -tz;
      const double mw = (typ == 0) ? mz : (typ == 1 ? tx : ty);
      const int wz = b;
      const int wx = ((bi + 1 == L) ? 0 : bi + 1) * L + bj;
      const int wy = bi * L + ((bj + 1 == L) ? 0 : bj + 1);
      if (wz <= w) row[wz] += mw * mz;
      if (wx <= w) row[wx] += mw * tx;
      if (wy <= w && !(open_cols && bj + 1 == L)) row[wy] += mw * ty;
    }
  }
  grp_sync<MULTI>(g);
  // Householder tridiagonalisation, column j: x = A[j+1:, j] -> alpha e_1 by
  // H = I - tau u u^T, u = x - alpha e_1.  Only the lower triangle of the
  // trailing block A22 (rows and columns j+1..N-1, m of them) is read and
  // updated; the product with A22 reads u from column j itself (u_0 = x_0 -
  // alpha, u_c = A[j+1+c][j]), which the step does not change, and stores it
  // in vv for the update.  Three group barriers per column: p = tau A22 u
  // with H lanes per row and, per warp, the partial of p^T u; then w = p -
  // (tau p^T u / 2) u; then A22 -= u w^T + w u^T, its first column (with
  // per-warp partials of the next step's s, the sum of squares below the
  // subdiagonal) and the rest of the packed triangle element by element over
  // the group's threads in the folded order of FoldWalk.  sc[0..31]: p^T u
  // partials, sc[32..63]: s.
  double* scP = wk.sc;
  double* scS = wk.sc + 32;
  double s;
  {
    double s0 = 0.0;
    for (int i = 2 + tid; i < N; i += nt) {
      const double a = A[tri(i, 0)];
      s0 = fma(a, a, s0);
    }
    s = grp_sum<MULTI>(s0, g, wk.sc);
  }
  for (int j = 0; j < N - 2; ++j) {
    const int m = N - j - 1, j1 = j + 1;
    const double x0 = A[tri(j1, j)];
    if (tid == 0) wk.d[j] = A[tri(j, j)];
    if (s == 0.0) {
      // column already reduced: no reflection; s of the next column directly
      if (tid == 0) wk.e[j] = x0;
      double s2 = 0.0;
      for (int i = j + 3 + tid; i < N; i += nt) {
        const double a = A[tri(i, j1)];
        s2 = fma(a, a, s2);
      }
      s = grp_sum<MULTI>(s2, g, wk.sc);
      continue;
    }
    const double nrm = sqrt(x0 * x0 + s);
    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
    const double u0 = x0 - alpha;
    const double tau = 2.0 / (u0 * u0 + s);
    if (tid == 0) wk.e[j] = alpha;
    // p_l = tau sum_c A22[l][c] u_c, u_c = A[tri(j1 + c, j)] (c >= 1): H lanes
    // of a warp per row (H = 1, 2, 4, .. while H m still fits the group), lane
    // h of a row taking the columns c = h mod H -- the row part c <= l
    // (contiguous), then the column part c > l -- alternately into two
    // accumulators, the H lanes' sums then added by a butterfly
    const int H = row_split(m, nt), h = lane & (H - 1);
    double part = 0.0;
    for (int l0 = 0; l0 < m; l0 += nt / H) {
      const int l = l0 + warp * (32 / H) + lane / H;
      double e0 = 0.0, e1 = 0.0;
      if (l < m) {
        const double* row = A + tri(j1 + l, j1);
        int c = h;
        if (c == 0) {
          e0 = row[0] * u0;
          c = H;
        }
        for (; c + H <= l; c += 2 * H) {
          e1 = fma(row[c], A[tri(j1 + c, j)], e1);
          e0 = fma(row[c + H], A[tri(j1 + c + H, j)], e0);
        }
        if (c <= l) {
          e1 = fma(row[c], A[tri(j1 + c, j)], e1);
          c += H;
        }
        for (; c + H < m; c += 2 * H) {
          const int b1 = tri(j1 + c, 0), b2 = tri(j1 + c + H, 0);
          e0 = fma(A[b1 + j1 + l], A[b1 + j], e0);
          e1 = fma(A[b2 + j1 + l], A[b2 + j], e1);
        }
        if (c < m) {
          const int b1 = tri(j1 + c, 0);
          e0 = fma(A[b1 + j1 + l], A[b1 + j], e0);
        }
      }
      double e = e0 + e1;
      for (int o = 1; o < H; o <<= 1) e += __shfl_xor_sync(kFull, e, o);
      if (l < m && h == 0) {
        const double p = tau * e, ul = l == 0 ? u0 : A[tri(j1 + l, j)];
        wk.pw[l] = p;
        wk.vv[l] = ul;
        part = fma(p, ul, part);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
    if (lane == 0) scP[warp] = part;
    grp_sync<MULTI>(g);
    double pv = 0.0;
    for (int w = 0; w < nw; ++w) pv += scP[w];
    const double Kc = 0.5 * tau * pv;
    for (int l = tid; l < m; l += nt) wk.pw[l] = fma(-Kc, wk.vv[l], wk.pw[l]);
    grp_sync<MULTI>(g);
    // A22 -= u w^T + w u^T (u in vv, w in pw): column 0 of A22 -- the next
    // step's column -- row r by thread r mod nt, with the partials of s; then
    // the rest of the packed triangle (rows and columns 1..m-1), in the
    // folded order of FoldWalk
    const double* uu = wk.vv;
    const double* ww = wk.pw;
    double sp = 0.0;
    for (int r = tid; r < m; r += nt) {
      double* a = A + tri(j1 + r, j1);
      const double x = fma(-uu[r], ww[0], fma(-ww[r], u0, *a));
      *a = x;
      if (r >= 2) sp = fma(x, x, sp);
    }
    const int ntri = (m - 1) * m / 2;
    FoldWalk fw(m - 1, tid, nt);
    for (int q = tid; q < ntri; q += nt, fw.next()) {
      int r, c;
      fw.rc(r, c);
      double* a = A + tri(j1 + 1 + r, j1 + 1 + c);
      *a = fma(-uu[r + 1], ww[c + 1], fma(-ww[r + 1], uu[c + 1], *a));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sp += __shfl_xor_sync(kFull, sp, o);
    if (lane == 0) scS[warp] = sp;
    grp_sync<MULTI>(g);
    s = 0.0;
    for (int w = 0; w < nw; ++w) s += scS[w];
  }
  if (tid == 0) {
    wk.d[N - 2] = A[tri(N - 2, N - 2)];
    wk.d[N - 1] = A[tri(N - 1, N - 1)];
    wk.e[N - 2] = A[tri(N - 1, N - 2)];
    wk.e[N - 1] = 0.0;
    // Gershgorin interval
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < N; ++i) {
      const double r = fabs(wk.e[i]) + (i > 0 ? fabs(wk.e[i - 1]) : 0.0);
      lo = fmin(lo, wk.d[i] - r);
      hi = fmax(hi, wk.d[i] + r);
    }
    wk.sc[0] = lo;
    wk.sc[1] = hi;
  }
  grp_sync<MULTI>(g);
  // squared off-diagonals for the Sturm recurrence (reuse vv), FP32 copies
  for (int i = tid; i < N; i += nt) {
    wk.vv[i] = wk.e[i] * wk.e[i];
    wk.d32[i] = (float)wk.d[i];
    wk.e32[i] = (float)(wk.e[i] * wk.e[i]);
  }
  const double glo = wk.sc[0], ghi = wk.sc[1];
  grp_sync<MULTI>(g);
  const EigGrid gr = eig_grid(wk, N, glo, ghi, tid, nt);
  grp_sync<MULTI>(g);
  double lp = 0.0, en = 0.0, cf = 0.0;
  for (int idx = tid; idx < N; idx += nt) {
    const double mu = fmax(eigen_idx(wk, gr, N, idx, glo, ghi), 0.0);
    const double eps = sqrt(mu);
    if (eps_out) eps_out[idx] = eps;
    thermal_add(eps, beta, lp, en, cf);
  }
  res[0] = grp_sum<MULTI>(lp, g, wk.sc);
  res[1] = grp_sum<MULTI>(en, g, wk.sc);
  res[2] = grp_sum<MULTI>(cf, g, wk.sc);
}

}  // namespace crbm
