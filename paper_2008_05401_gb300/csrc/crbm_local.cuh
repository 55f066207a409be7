// Local-update Metropolis sweeps (the paper's baselines, Sec. III and IV),
// run by the fused kernel in mode 3 with the lattices resident in shared memory.
//
// Ising, checkerboard: the sites with (i + j) even, then the odd ones (even L,
// so the sites of one colour never neighbour each other); site (i, j) with u
// unequal neighbours flips iff u_site < e^{-beta dE}, dE = 2 J (4 - 2u).
// Kitaev: sites n = 0 .. N-1 in order; eta_n flips iff
// log u_site < log pi(eta with eta_n flipped) - log pi(eta), each proposal
// needing one eigen-stage.  The uniform of site n is word n % 4 of Philox
// block n / 4 of tag kTagLocal at the sweep's step.
#pragma once
#include "crbm_device.cuh"
#include "crbm_df64.cuh"

namespace crbm {

// Number of ones and of unequal nearest-neighbour pairs (Ising) or of
// hexagons with flux -1 (Kitaev) of lattice v: per-thread partials.
__device__ inline void lattice_counts(const JobDev& jb, const Grp& g, const uint32_t* v, double (&out)[2]) {
  const int L = jb.L, N = jb.N;
  int ones = 0, pairs = 0;
  if (g.active) {
    for (int n = g.r; n < N; n += g.tpc) {
      const int i = n / L, j = n - i * L;
      const uint32_t b0 = site_bit(v, n);
      ones += (int)b0;
      if (jb.kind == kIsing) {
        pairs += (int)(b0 ^ site_bit(v, i * L + (j + 1 == L ? 0 : j + 1)));
        pairs += (int)(b0 ^ site_bit(v, (i + 1 == L ? 0 : i + 1) * L + j));
      } else {
        // the hexagon of cell r holds the z-bonds r and r - e1 + e2 (none in
        // column L-1 when the columns are open)
        const int i2 = (i == 0) ? L - 1 : i - 1, j2 = (j + 1 == L) ? 0 : j + 1;
        if (!(jb.lc_edge && j + 1 == L)) pairs += (int)(b0 ^ site_bit(v, i2 * L + j2));
      }
    }
  }
  out[0] = (double)ones;
  out[1] = (double)pairs;
}

// One colour of a checkerboard sweep of the group's lattice v (in place).
// thr[u] = e^{-beta dE(u)} 2^32: accept iff word + 1/2 < thr[u], which is
// u_site < e^{-beta dE} exactly (scaling by 2^32 is exact).
__device__ inline unsigned ising_colour(const JobDev& jb, const Grp& g, uint32_t* v, uint32_t step, int colour,
                                        const double* thr) {
  const int L = jb.L, N = jb.N, nblk = (N + 3) >> 2;
  unsigned nacc = 0;
  if (!g.active) return 0;
  for (int q = g.r; q < nblk; q += g.tpc) {
    const uint4 w = philox4x32_10_rk(make_uint4((uint32_t)q, kTagLocal, step, g.cid), jb.rk);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int n = 4 * q + t;
      if (n >= N) break;
      const int i = n / L, j = n - i * L;
      if (((i + j) & 1) != colour) continue;
      const uint32_t s0 = site_bit(v, n);
      const int iu = (i == 0) ? L - 1 : i - 1, id = (i + 1 == L) ? 0 : i + 1;
      const int jl = (j == 0) ? L - 1 : j - 1, jr = (j + 1 == L) ? 0 : j + 1;
      const int u = (int)(s0 ^ site_bit(v, iu * L + j)) + (int)(s0 ^ site_bit(v, id * L + j)) +
                    (int)(s0 ^ site_bit(v, i * L + jl)) + (int)(s0 ^ site_bit(v, i * L + jr));
      if ((double)pick(w, t) + 0.5 < thr[u]) {
        atomicXor(&v[n >> 5], 1u << (n & 31));
        ++nacc;
      }
    }
  }
  return nacc;
}

}  // namespace crbm
