// Fused CRBM proposal + Metropolis-Hastings kernel (one launch runs S
// proposals; lattices stay in shared memory for the whole launch).
//
// Per proposal and chain (arXiv:2008.05401):
//   g x [hidden half-step (Eq. B2), visible half-step (Eq. B3)]   -> v'
//   F(v') (Eq. 13) and the lattice sums of v'
//   log pi(v'): Ising -beta E (Eq. 14) | Kitaev sum log 2cosh(beta eps/2) (Sec. IV)
//   log r = [log pi(v') - log pi(v)] + [F(v') - F(v)], accept iff log u < log r
//   (Eq. B5 with the pair (pi, P_CRBM); the Gibbs kernel is reversible w.r.t.
//   P_CRBM, App. B.1), then observables of the state after the decision.
// Template parameters: model kind, precision, and K, k fixed at compile time
// for the common filter banks (0 = runtime values).
#pragma once
#include "crbm_device.cuh"
#include "crbm_df64.cuh"
#include "crbm_local.cuh"
#include "crbm_kernels.h"

namespace crbm {

struct ChainSm {
  double F, Fb, lp, E;
  double ot[kNobs];      // observables of the current lattice
  double os[kNobs];      // running sums
  double Fp, Bp, lpp, Ep;
  double lpb, lppb;      // bounds on |log pi - FP64 path's log pi| (current, proposed)
  double otp[kNobs];
  double beta;
  double thr[5];         // local Ising sweeps: e^{-beta dE} 2^32 for 0..4 unequal neighbours
  double logu;           // tensor-core kernel: log u of the current proposal's MH draw
  double cst, mgs;       // tensor-core kernel: the tile's constant margin terms, the
                         // current state's margin terms (both off the MH thread's path)
  unsigned long long acc, rec, rec_mh;
  int cur, flag_rec, flag_acc, onesp;   // onesp: set units of the proposal (tensor-core kernel)
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared-memory work areas of one Kitaev chain (one per thread group of the
// CTA): the packed lower triangle of A (N (N+1) / 2 FP64 or double-FP32
// entries), d, e, vv, pw (N each), 64 doubles of reduction scratch, the FP32
// tridiagonal copies (N each) and the proposed spectrum of a local sweep (N).
__host__ __device__ inline size_t kitaev_work_bytes(int N) {
  const size_t n = (size_t)N;
  return align16(n * (n + 1) / 2 * 8) + 4 * align16(n * 8) + align16(64 * 8) + 2 * align16(n * 4) + align16(n * 8);
}

// The mixed path's FP64 free energy (rare), out of line to spare registers.
static __device__ __noinline__ void free_energy64(const JobDev& jb, const Tabs& tb, const Grp& g,
                                                  const uint32_t* v, double* out) {
  double o[4];
  free_phase<kFP64, 0, 0>(jb, tb, g, v, o);
  for (int i = 0; i < 4; ++i) out[i] = o[i];
}

// FP64 free energy, log pi, E and observables of chain c's lattice from the
// group sums fo (Eq. 13 sums, magnetisation count, bond/vison count) and, for
// the Kitaev kind, kr = (log pi, e, c_f) of its spectrum.
template <int KIND>
// Fb: bound on |F - F_fp64| of an FP32 free energy (0 for an FP64 one).
__device__ inline void store_evaluation(const JobDev& jb, int c, double beta, const double* fo, const double* kr,
                                        double Fb = 0.0) {
  const int N = jb.N;
  const double Fv = -jb.vb * fo[2] - fo[0];
  double lp, E, ot[kNobs];
  if (KIND == kIsing) {
    E = -jb.J[0] * (double)(2 * N - 2 * (int)fo[3]);
    const double M = 2.0 * fo[2] - (double)N;
    lp = -beta * E;
    ot[0] = E; ot[1] = E * E; ot[2] = fabs(M); ot[3] = M * M;
  } else {
    lp = kr[0];
    E = kr[1];
    ot[0] = kr[1]; ot[1] = kr[1] * kr[1]; ot[2] = kr[2]; ot[3] = fo[3] / (double)jb.nhex;
  }
  jb.F[c] = Fv;
  jb.Fb[c] = Fb;
  jb.Lb[c] = 0.0;
  jb.logpi[c] = lp;
  jb.Ephys[c] = E;
  for (int o = 0; o < kNobs; ++o) jb.obs_t[(size_t)c * kNobs + o] = ot[o];
}

// AUX = 0: the proposal loop (mode 0) only; AUX = 1: modes 1-3.  Two kernels,
// so that the hot proposal loop carries none of the other modes' code and
// registers (with them it spilled).  MULTI (Kitaev, mode 0 only): CTAs hold
// several chain groups, which synchronise on named barriers of their own;
// without it every CTA holds one chain and uses the CTA barrier only.
template <int KIND, int PREC, int KC, int kC, int NT, int AUX, bool MULTI = false>
__global__ void __launch_bounds__(NT, CRBM_MIN_BLOCKS * 256 / NT) crbm_step_kernel(const __grid_constant__ LaunchParams prm) {
  int jid = 0;
  while (jid + 1 < prm.n_jobs && (int)blockIdx.x >= prm.tile_begin[jid + 1]) ++jid;
  const JobDev& jb = prm.job[jid];
  const int ltile = (int)blockIdx.x - prm.tile_begin[jid];
  const int tid = threadIdx.x;
  const int N = jb.N, P = jb.P, K = jb.K, T = 1 << jb.k, nlut = jb.ncls * K * jb.k * T;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* sp = smem_raw;
  Tabs tb;
  tb.T = T;
  tb.f64 = tb.b64 = nullptr;
  tb.fd = tb.bd = tb.fh = tb.fl = nullptr;
  tb.fd4 = tb.fh4 = tb.fl4 = nullptr;
  const int nq = jb.k * T;   // entries of a filter-interleaved table
  double* t64[2] = {nullptr, nullptr};
  float* t32[4] = {nullptr, nullptr, nullptr, nullptr};
  float4* t4[3] = {nullptr, nullptr, nullptr};
  if (PREC == kFP64) {
    for (int i = 0; i < 2; ++i) {
      t64[i] = (double*)sp;
      sp += align16((size_t)nlut * 8);
    }
    tb.f64 = t64[0];
    tb.b64 = t64[1];
  } else if (KC == 4) {
    for (int i = 0; i < 3; ++i) {
      t4[i] = (float4*)sp;
      sp += align16((size_t)nq * 16 * 8);      // 8 bank-interleaved copies
    }
    t32[1] = (float*)sp;
    sp += align16((size_t)nlut * 4);
    tb.fd4 = t4[0] + (threadIdx.x & 7);
    tb.fh4 = t4[1] + (threadIdx.x & 7);
    tb.fl4 = t4[2] + (threadIdx.x & 7);
    tb.bd = t32[1];
  } else {
    for (int i = 0; i < 4; ++i) {
      t32[i] = (float*)sp;
      sp += align16((size_t)nlut * 4);
    }
    tb.fd = t32[0];
    tb.bd = t32[1];
    tb.fh = t32[2];
    tb.fl = t32[3];
  }
  ChainSm* cs = (ChainSm*)sp;
  sp += align16(jb.nc * sizeof(ChainSm));
  double* scratch = (double*)sp;
  sp += align16(64 * 8);
  unsigned char* kwork = sp;     // Kitaev: the work areas of the CTA's nc chains
  if (KIND == kKitaev) sp += (size_t)jb.nc * kitaev_work_bytes(N);
  uint32_t* planes = (uint32_t*)sp;

  Grp g;
  g.tpc = NT / jb.nc;
  g.gl = tid / g.tpc;
  g.r = tid - g.gl * g.tpc;
  g.c = ltile * jb.nc + g.gl;
  g.active = g.c < jb.n_chains;
  g.cid = (uint32_t)(jb.cid_base + (uint64_t)g.c);
  KitaevWork wk;
  double* eps_st = nullptr;     // Kitaev local sweeps: spectrum of the proposed lattice
  if (KIND == kKitaev) {
    unsigned char* kp = MULTI ? kwork + (size_t)g.gl * kitaev_work_bytes(N) : kwork;
    wk.A = (double*)kp;
    kp += align16((size_t)N * (N + 1) / 2 * 8);
    wk.d = (double*)kp;
    kp += align16((size_t)N * 8);
    wk.e = (double*)kp;
    kp += align16((size_t)N * 8);
    wk.vv = (double*)kp;
    kp += align16((size_t)N * 8);
    wk.pw = (double*)kp;
    kp += align16((size_t)N * 8);
    wk.sc = (double*)kp;
    kp += align16(64 * 8);
    wk.d32 = (float*)kp;
    kp += align16((size_t)N * 4);
    wk.e32 = (float*)kp;
    kp += align16((size_t)N * 4);
    eps_st = (double*)kp;
  }
  uint32_t* my = planes + (size_t)g.gl * (2 + K) * P;
  ChainSm& ch = cs[g.gl];

  for (int i = tid; i < nlut; i += NT) {
    if (PREC == kFP64) {
      t64[0][i] = jb.f64[i];
      t64[1][i] = jb.b64[i];
    } else if (KC == 4) {
      t32[1][i] = jb.bd[i];
    } else {
      t32[0][i] = jb.fd[i];
      t32[1][i] = jb.bd[i];
      t32[2][i] = jb.fh[i];
      t32[3][i] = jb.fl[i];
    }
  }
  if (PREC == kMixed && KC == 4) {
    for (int i = tid; i < nq * 8; i += NT) {
      t4[0][i] = jb.fd4[i >> 3];
      t4[1][i] = jb.fh4[i >> 3];
      t4[2][i] = jb.fl4[i >> 3];
    }
  }
  for (int i = tid; i < jb.nc * (2 + K) * P; i += NT) planes[i] = 0u;
  __syncthreads();
  if (g.r == 0) {
    // every slot, including the unused slots of a partial last tile, starts
    // from a defined state: the plane index `cur` addresses shared memory
    ch.F = ch.Fb = ch.lp = ch.E = 0.0;
    ch.lpb = ch.lppb = 0.0;
    for (int o = 0; o < kNobs; ++o) ch.ot[o] = ch.os[o] = 0.0;
    ch.beta = 1.0;
    ch.acc = 0ull;
    ch.rec = 0ull;
    ch.rec_mh = 0ull;
    ch.cur = 0;
    ch.flag_rec = 0;
    ch.flag_acc = 0;
  }
  if (g.active) {
    for (int w = g.r; w < jb.Wd; w += g.tpc) my[w] = jb.bits[(size_t)g.c * jb.Wd + w];
    if (g.r == 0) {
      ch.F = jb.F[g.c];
      ch.Fb = jb.Fb[g.c];
      ch.lpb = jb.Lb[g.c];
      ch.lp = jb.logpi[g.c];
      ch.E = jb.Ephys[g.c];
      for (int o = 0; o < kNobs; ++o) {
        ch.ot[o] = jb.obs_t[(size_t)g.c * kNobs + o];
        // sums continue in place: the same sequence of additions however a
        // run is split into launches or batched with other jobs
        ch.os[o] = jb.obs[(size_t)g.c * kNobs + o];
      }
      ch.beta = 1.0 / jb.T[g.c];
    }
  }
  __syncthreads();
  unsigned nrec = 0;

  if (AUX && prm.mode == 1) {
    // evaluate F (FP64, or in the mixed path FP32 with its certified bound,
    // as after a mixed proposal), log pi and the observables (FP64) of the
    // current lattices
    double fo[4];
    if (PREC == kMixed) free_phase<PREC, KC, kC>(jb, tb, g, my, fo);
    else free_energy64(jb, tb, g, my, fo);
    grp_reduce<4>(fo, g, scratch);
    double kr[3] = {0.0, 0.0, 0.0};
    if (KIND == kKitaev)
      kitaev_logpi64<MULTI>(g, my, jb.L, jb.J, g.active ? ch.beta : 1.0, wk, kr,
                     g.active ? jb.eps + (size_t)g.c * N : nullptr, jb.lc_edge > 0);
    if (g.active && g.r == 0) {
      double Fb = 0.0;
      if (PREC == kMixed) {
        const double Fv = -jb.vb * fo[2] - fo[0];
        Fb = fo[1] + (double)K * (double)N * (1.5 * 0x1p-23 + (double)jb.csp) + 1e-12 * fabs(Fv);
      }
      store_evaluation<KIND>(jb, g.c, ch.beta, fo, kr, Fb);
    }
    return;
  }

  if (AUX && prm.mode == 2) {
    // tempering: the RBM chain makes g Gibbs steps without correction (Eq. B4),
    // then its new lattice y' and the physical chain x of the same slot (job
    // prm.job[1]) are exchanged with the Eq. (B5) probability for the pair
    // (pi, P_CRBM):  log a = [log pi(y') - log pi(x)] + [F(y') - F(x)].  In the
    // mixed path F(y') is the FP32 value with its certified bound and F(x) may
    // carry one too; a decision inside the bounds is redone with FP64 F.
    const JobDev& xj = prm.job[1];
    const uint32_t step = (uint32_t)*(volatile unsigned long long*)jb.step;
    const uint32_t cycle = (uint32_t)*(volatile unsigned long long*)xj.step;
    uint32_t* vp = my + P;
    uint32_t* h = my + 2 * P;
    const uint32_t* src = my;
    for (int sub = 0; sub < prm.g; ++sub) {
      hidden_phase<PREC, KC, kC>(jb, tb, g, src, h, P, step, sub, nrec);
      __syncthreads();
      visible_phase<PREC, KC, kC>(jb, tb, g, h, vp, P, step, sub, nrec);
      __syncthreads();
      src = vp;
    }
    double fo[4];
    free_phase<PREC, KC, kC>(jb, tb, g, vp, fo);
    grp_reduce<4>(fo, g, scratch);
    double kr[3] = {0.0, 0.0, 0.0};
    if (KIND == kKitaev)
      kitaev_logpi64<MULTI>(g, vp, jb.L, jb.J, g.active ? ch.beta : 1.0, wk, kr,
                     g.active ? jb.eps + (size_t)g.c * N : nullptr, jb.lc_edge > 0);
    // the physical chain's lattice into the first hidden plane (free now)
    if (g.active)
      for (int w = g.r; w < jb.Wd; w += g.tpc) h[w] = xj.bits[(size_t)g.c * jb.Wd + w];
    if (g.active && g.r == 0) {
      ch.Fp = -jb.vb * fo[2] - fo[0];
      ch.Bp = (PREC == kMixed)
                  ? fo[1] + (double)K * (double)N * (1.5 * 0x1p-23 + (double)jb.csp) + 1e-12 * fabs(ch.Fp)
                  : 0.0;
      if (KIND == kIsing) {
        const double E = -jb.J[0] * (double)(2 * N - 2 * (int)fo[3]);
        const double M = 2.0 * fo[2] - (double)N;
        ch.Ep = E;
        ch.lpp = -ch.beta * E;
        ch.otp[0] = E; ch.otp[1] = E * E; ch.otp[2] = fabs(M); ch.otp[3] = M * M;
      } else {
        ch.Ep = kr[1];
        ch.lpp = kr[0];
        ch.otp[0] = kr[1]; ch.otp[1] = kr[1] * kr[1]; ch.otp[2] = kr[2]; ch.otp[3] = fo[3] / (double)jb.nhex;
      }
      ch.F = xj.F[g.c];
      ch.Fb = xj.Fb[g.c];
      ch.lp = xj.logpi[g.c];
      const double loga = (ch.lpp - ch.lp) + (ch.Fp - ch.F);
      const uint4 w = philox4x32_10_rk(make_uint4(0u, kTagSwap, cycle, (uint32_t)(xj.cid_base + (uint64_t)g.c)),
                                       xj.rk);
      const double logu = log(((double)w.x + 0.5) * 0x1p-32);
      ch.flag_rec = 0;
      if (PREC == kFP64) {
        ch.flag_acc = logu < loga;
      } else {
        const double Mg = ch.Bp + ch.Fb + 1e-12 * (fabs(ch.lpp) + fabs(ch.lp) + fabs(ch.Fp) + fabs(ch.F)) + 1e-300;
        if (loga - logu > Mg) ch.flag_acc = 1;
        else if (logu - loga > Mg) ch.flag_acc = 0;
        else ch.flag_rec = 1;
      }
    }
    if (PREC == kMixed) {
      const int need = __syncthreads_or(g.active && g.r == 0 && ch.flag_rec);
      if (need) {
        // FP64 free energies of y' and (when only its FP32 value is known) of x
        Tabs tb64g = tb;
        tb64g.f64 = jb.f64;
        tb64g.b64 = jb.b64;
        Grp g2 = g;
        g2.active = g.active && ch.flag_rec;
        double f1[4];
        free_energy64(jb, tb64g, g2, vp, f1);
        grp_reduce<4>(f1, g2, scratch);
        Grp g3 = g2;
        g3.active = g2.active && ch.Fb != 0.0;
        double f2[4];
        free_energy64(jb, tb64g, g3, h, f2);
        grp_reduce<4>(f2, g3, scratch);
        if (g2.active && g.r == 0) {
          ch.Fp = -jb.vb * f1[2] - f1[0];
          ch.Bp = 0.0;
          if (g3.active) {
            ch.F = -jb.vb * f2[2] - f2[0];
            ch.Fb = 0.0;
          }
          const double loga = (ch.lpp - ch.lp) + (ch.Fp - ch.F);
          const uint4 w = philox4x32_10_rk(
              make_uint4(0u, kTagSwap, cycle, (uint32_t)(xj.cid_base + (uint64_t)g.c)), xj.rk);
          ch.flag_acc = log(((double)w.x + 0.5) * 0x1p-32) < loga;
          ch.rec_mh += 1ull;
        }
      }
    }
    if (nrec) atomicAdd(&ch.rec, (unsigned long long)nrec);
    __syncthreads();
    if (g.active) {
      const bool sw = ch.flag_acc != 0;
      const size_t c = (size_t)g.c;
      uint32_t* xb = xj.bits + c * jb.Wd;
      uint32_t* yb = jb.bits + c * jb.Wd;
      for (int w = g.r; w < jb.Wd; w += g.tpc) {
        if (sw) {
          xb[w] = vp[w];
          yb[w] = h[w];
        } else {
          yb[w] = vp[w];
        }
      }
      if (KIND == kKitaev && sw) {
        for (int l = g.r; l < N; l += g.tpc) {
          const double t = xj.eps[c * N + l];
          xj.eps[c * N + l] = jb.eps[c * N + l];
          jb.eps[c * N + l] = t;
        }
      }
      if (g.r == 0) {
        if (sw) {
          // the RBM slot takes x (read before the physical slot is overwritten)
          jb.F[c] = ch.F;
          jb.Fb[c] = ch.Fb;
          jb.Lb[c] = xj.Lb[c];
          jb.logpi[c] = ch.lp;
          jb.Ephys[c] = xj.Ephys[c];
          for (int o = 0; o < kNobs; ++o) jb.obs_t[c * kNobs + o] = xj.obs_t[c * kNobs + o];
          xj.F[c] = ch.Fp;
          xj.Fb[c] = ch.Bp;
          xj.Lb[c] = 0.0;
          xj.logpi[c] = ch.lpp;
          xj.Ephys[c] = ch.Ep;
          for (int o = 0; o < kNobs; ++o) xj.obs_t[c * kNobs + o] = ch.otp[o];
          xj.acc[c] += 1ull;
        } else {
          jb.F[c] = ch.Fp;
          jb.Fb[c] = ch.Bp;
          jb.Lb[c] = 0.0;
          jb.logpi[c] = ch.lpp;
          jb.Ephys[c] = ch.Ep;
          for (int o = 0; o < kNobs; ++o) jb.obs_t[c * kNobs + o] = ch.otp[o];
        }
        jb.rec[2 * c] += ch.rec;
        jb.rec[2 * c + 1] += ch.rec_mh;
      }
    }
    return;
  }

  if (AUX && prm.mode == 3) {
    // local-update Metropolis sweeps (Sec. III, Sec. IV baselines)
    const unsigned long long step0 = *(volatile unsigned long long*)jb.step;
    if (KIND == kIsing && g.active && g.r == 0) {
      for (int u = 0; u < 5; ++u) {
        const double dE = (2.0 * jb.J[0]) * (double)(4 - 2 * u);
        ch.thr[u] = exp(-ch.beta * dE) * 0x1p32;
      }
    }
    __syncthreads();
    unsigned nacc = 0;
    for (int s = 0; s < prm.S; ++s) {
      const uint32_t step = (uint32_t)(step0 + (uint64_t)s);
      if (KIND == kIsing) {
        uint32_t* v = my + ch.cur * P;
        nacc += ising_colour(jb, g, v, step, 0, ch.thr);
        __syncthreads();
        nacc += ising_colour(jb, g, v, step, 1, ch.thr);
        __syncthreads();
      } else {
        // per chain group: every branch below is uniform in the group, and only
        // the group synchronises (a short last tile has groups without a chain)
        for (int n = 0; n < N; ++n) {
          const uint32_t* v = my + ch.cur * P;
          uint32_t* vp = my + (ch.cur ^ 1) * P;
          for (int w = g.r; w < jb.Wd; w += g.tpc) vp[w] = v[w] ^ ((w == (n >> 5)) ? (1u << (n & 31)) : 0u);
          grp_sync<MULTI>(g);
          double kr[4] = {0.0, 0.0, 0.0, 0.0};
          if (PREC == kMixed) {
            kitaev_logpi_df<MULTI>(g, vp, jb.L, jb.J, ch.beta, wk, kr, jb.lc_edge > 0);
          } else {
            double k3[3];
            kitaev_logpi64<MULTI>(g, vp, jb.L, jb.J, ch.beta, wk, k3, eps_st, jb.lc_edge > 0);
            kr[0] = k3[0];
            kr[1] = k3[1];
            kr[2] = k3[2];
          }
          if (g.r == 0) {
            const uint4 w = philox4x32_10_rk(make_uint4((uint32_t)(n >> 2), kTagLocal, step, g.cid), jb.rk);
            const double logu = log(((double)pick(w, n & 3) + 0.5) * 0x1p-32);
            const double logr = kr[0] - ch.lp;
            ch.lpp = kr[0];
            ch.lppb = kr[3];
            ch.Ep = kr[1];
            ch.otp[0] = kr[1]; ch.otp[1] = kr[1] * kr[1]; ch.otp[2] = kr[2];
            ch.flag_rec = 0;
            if (PREC == kFP64) {
              ch.flag_acc = logu < logr;
            } else {
              const double M = ch.lppb + ch.lpb + 1e-12 * (fabs(ch.lpp) + fabs(ch.lp)) + 1e-300;
              if (logr - logu > M) ch.flag_acc = 1;
              else if (logu - logr > M) ch.flag_acc = 0;
              else ch.flag_rec = 1;
            }
          }
          grp_sync<MULTI>(g);
          if (PREC == kMixed && ch.flag_rec) {
            // the FP64 eigen-stage of the proposal (and of the current lattice
            // when its log-weight came from the df64 stage)
            double k1v[3], k0v[3] = {0.0, 0.0, 0.0};
            const bool redo_v = ch.lpb != 0.0;
            kitaev_logpi64<MULTI>(g, vp, jb.L, jb.J, ch.beta, wk, k1v, eps_st, jb.lc_edge > 0);
            if (redo_v) kitaev_logpi64<MULTI>(g, v, jb.L, jb.J, ch.beta, wk, k0v, nullptr, jb.lc_edge > 0);
            if (g.r == 0) {
              ch.lpp = k1v[0];
              ch.lppb = 0.0;
              ch.Ep = k1v[1];
              ch.otp[0] = k1v[1]; ch.otp[1] = k1v[1] * k1v[1]; ch.otp[2] = k1v[2];
              if (redo_v) {
                ch.lp = k0v[0];
                ch.lpb = 0.0;
              }
              const uint4 w = philox4x32_10_rk(make_uint4((uint32_t)(n >> 2), kTagLocal, step, g.cid), jb.rk);
              const double logu = log(((double)pick(w, n & 3) + 0.5) * 0x1p-32);
              ch.flag_acc = logu < ch.lpp - ch.lp;
              ch.rec_mh += 1ull;
            }
            grp_sync<MULTI>(g);
          }
          if (ch.flag_acc) {
            // the spectrum cache follows the lattice when the proposal's came from the FP64 stage
            if (g.active && (PREC == kFP64 || ch.flag_rec))
              for (int l = g.r; l < N; l += g.tpc) jb.eps[(size_t)g.c * N + l] = eps_st[l];
            grp_sync<MULTI>(g);
            if (g.r == 0) {
              ch.cur ^= 1;
              ch.lp = ch.lpp;
              ch.lpb = ch.lppb;
              ch.E = ch.Ep;
              for (int o = 0; o < 3; ++o) ch.ot[o] = ch.otp[o];
              ch.acc += 1ull;
            }
          }
          grp_sync<MULTI>(g);
        }
      }
      // observables of the lattice after the sweep
      double cn[2];
      lattice_counts(jb, g, my + ch.cur * P, cn);
      grp_reduce<2>(cn, g, scratch);
      if (g.active && g.r == 0) {
        if (KIND == kIsing) {
          const double E = -jb.J[0] * (double)(2 * N - 2 * (int)cn[1]);
          const double M = 2.0 * cn[0] - (double)N;
          ch.E = E;
          ch.lp = -ch.beta * E;
          ch.ot[0] = E; ch.ot[1] = E * E; ch.ot[2] = fabs(M); ch.ot[3] = M * M;
        } else {
          ch.ot[3] = cn[1] / (double)jb.nhex;
        }
        if (prm.correct) {
          for (int o = 0; o < kNobs; ++o) ch.os[o] += ch.ot[o];
          trace_store(jb, g.c, step0 + (uint64_t)s, ch.E);
        }
      }
      __syncthreads();
    }
    if (nacc) atomicAdd(&ch.acc, (unsigned long long)nacc);
    __syncthreads();
    // FP64 free energy of the final lattices, then everything back to the job
    Tabs tb64 = tb;
    tb64.f64 = jb.f64;
    tb64.b64 = jb.b64;
    double fo[4];
    free_energy64(jb, tb64, g, my + ch.cur * P, fo);
    grp_reduce<4>(fo, g, scratch);
    if (g.active) {
      const uint32_t* v = my + ch.cur * P;
      for (int w = g.r; w < jb.Wd; w += g.tpc) jb.bits[(size_t)g.c * jb.Wd + w] = v[w];
      if (g.r == 0) {
        jb.F[g.c] = -jb.vb * fo[2] - fo[0];
        jb.Fb[g.c] = 0.0;
        jb.Lb[g.c] = ch.lpb;
        jb.logpi[g.c] = ch.lp;
        jb.Ephys[g.c] = ch.E;
        for (int o = 0; o < kNobs; ++o) {
          jb.obs_t[(size_t)g.c * kNobs + o] = ch.ot[o];
          jb.obs[(size_t)g.c * kNobs + o] = ch.os[o];
        }
        jb.acc[g.c] += ch.acc;
        jb.rec[2 * (size_t)g.c + 1] += ch.rec_mh;
      }
    }
    return;
  }

  if (AUX) return;
  // The Kitaev kind's chain groups are warp-aligned and independent inside
  // the proposal loop: they synchronise and reduce on their own (a group whose
  // eigen-stage takes longer holds back no other chain of the CTA); the Ising
  // kind's groups may be smaller than a warp and use the CTA barrier.
  auto loop_sync = [&]() {
    if (KIND == kKitaev && MULTI) grp_sync<MULTI>(g);
    else __syncthreads();
  };
  auto loop_reduce4 = [&](double (&x)[4], const Grp& gg) {
    if (KIND == kKitaev && MULTI) grp_reduce_local<4, MULTI>(x, gg, wk.sc);
    else grp_reduce<4>(x, gg, scratch);
  };
  const uint32_t k0 = (uint32_t)jb.seed, k1 = (uint32_t)(jb.seed >> 32);
  // the step counter lives in device memory (advanced by advance_steps after
  // the launch), so a captured CUDA graph can be replayed
  const unsigned long long step0 = *(volatile unsigned long long*)jb.step;
  for (int s = 0; s < prm.S; ++s) {
    const uint32_t step = (uint32_t)(step0 + (uint64_t)s);
    const int cur = ch.cur;
    uint32_t* v = my + cur * P;
    uint32_t* vp = my + (cur ^ 1) * P;
    uint32_t* h = my + 2 * P;
    const uint32_t* src = v;
    for (int sub = 0; sub < prm.g; ++sub) {
      hidden_phase<PREC, KC, kC>(jb, tb, g, src, h, P, step, sub, nrec);
      loop_sync();
      visible_phase<PREC, KC, kC>(jb, tb, g, h, vp, P, step, sub, nrec);
      loop_sync();
      src = vp;
    }
    double fo[4];
    free_phase<PREC, KC, kC>(jb, tb, g, vp, fo);
    loop_reduce4(fo, g);
    double kr[4] = {0.0, 0.0, 0.0, 0.0};
    if (KIND == kKitaev) {
      if (PREC == kMixed) {
        kitaev_logpi_df<MULTI>(g, vp, jb.L, jb.J, g.active ? ch.beta : 1.0, wk, kr, jb.lc_edge > 0);
      } else {
        double k3[3];
        kitaev_logpi64<MULTI>(g, vp, jb.L, jb.J, g.active ? ch.beta : 1.0, wk, k3, nullptr, jb.lc_edge > 0);
        kr[0] = k3[0];
        kr[1] = k3[1];
        kr[2] = k3[2];
      }
    }
    double logu = 0.0;
    if (g.active && g.r == 0) {
      if (KIND == kIsing) {
        const double E = -jb.J[0] * (double)(2 * N - 2 * (int)fo[3]);
        const double M = 2.0 * fo[2] - (double)N;
        ch.Ep = E;
        ch.lpp = -ch.beta * E;
        ch.otp[0] = E; ch.otp[1] = E * E; ch.otp[2] = fabs(M); ch.otp[3] = M * M;
      } else {
        ch.Ep = kr[1];
        ch.lpp = kr[0];
        ch.otp[0] = kr[1]; ch.otp[1] = kr[1] * kr[1]; ch.otp[2] = kr[2]; ch.otp[3] = fo[3] / (double)jb.nhex;
      }
      ch.lppb = kr[3];
      ch.Fp = -jb.vb * fo[2] - fo[0];
      ch.Bp = (PREC == kMixed)
                  ? fo[1] + (double)K * (double)N * (1.5 * 0x1p-23 + (double)jb.csp) + 1e-12 * fabs(ch.Fp)
                  : 0.0;
      ch.flag_rec = 0;
      if (!prm.correct) {
        ch.flag_acc = 1;
      } else {
        const double logr = (ch.lpp - ch.lp) + (ch.Fp - ch.F);
        const uint4 w = philox4x32_10_rk(make_uint4(0u, kTagAcc, step, g.cid), jb.rk);
        logu = log(((double)w.x + 0.5) * 0x1p-32);
        if (PREC == kFP64) {
          ch.flag_acc = logu < logr;
        } else {
          const double M = ch.Bp + ch.Fb + ch.lppb + ch.lpb +
                           1e-12 * (fabs(ch.lpp) + fabs(ch.lp) + fabs(ch.Fp) + fabs(ch.F)) + 1e-300;
          if (logr - logu > M) ch.flag_acc = 1;
          else if (logu - logr > M) ch.flag_acc = 0;
          else ch.flag_rec = 1;
        }
      }
    }
    if (PREC == kMixed && KIND == kIsing) {
      // second level: F of v' (and of v when only an FP32 value of it is
      // known) with df64 softplus (bound ~1e-7); flag_rec = 2 sends a decision
      // that still straddles the threshold on to the FP64 path's code below
      if (__syncthreads_or(g.active && g.r == 0 && ch.flag_rec)) {
        Grp g2 = g;
        g2.active = g.active && ch.flag_rec;
        Grp g3 = g2;
        g3.active = g2.active && ch.Fb != 0.0;
        double f1[3], f2[3];
        free_sum_df<KC ? KC : kMaxK>(jb, g2, vp, f1);
        grp_reduce<3>(f1, g2, scratch);
        free_sum_df<KC ? KC : kMaxK>(jb, g3, v, f2);
        grp_reduce<3>(f2, g3, scratch);
        if (g2.active && g.r == 0) {
          ch.Fp = -jb.vb * f1[2] - f1[0];
          ch.Bp = f1[1] + 1e-15 * fabs(ch.Fp);
          if (g3.active) {
            ch.F = -jb.vb * f2[2] - f2[0];
            ch.Fb = f2[1] + 1e-15 * fabs(ch.F);
          }
          const double logr = (ch.lpp - ch.lp) + (ch.Fp - ch.F);
          const uint4 w = philox4x32_10_rk(make_uint4(0u, kTagAcc, step, g.cid), jb.rk);
          const double lu = log(((double)w.x + 0.5) * 0x1p-32);
          const double Mg = ch.Bp + ch.Fb + 1e-12 * (fabs(ch.lpp) + fabs(ch.lp) + fabs(ch.Fp) + fabs(ch.F)) + 1e-300;
          if (logr - lu > Mg) ch.flag_acc = 1, ch.flag_rec = 0;
          else if (lu - logr > Mg) ch.flag_acc = 0, ch.flag_rec = 0;
          else ch.flag_rec = 2;
          ch.rec_mh += 1ull;
        }
      }
    }
    if (PREC == kMixed) {
      int need;
      if (KIND == kKitaev && MULTI) {
        loop_sync();                 // the leader's flag_rec, read by its whole group
        need = g.active && ch.flag_rec;
      } else {
        need = __syncthreads_or(g.active && g.r == 0 && ch.flag_rec);
      }
      if (need) {
        // the FP64 path's free energies of v' (and of v when only its FP32
        // value is known), computed by the same code and reduction order
        // FP64 tables from global memory (the mixed kernel keeps only FP32 ones)
        Tabs tb64g = tb;
        tb64g.f64 = jb.f64;
        tb64g.b64 = jb.b64;
        Grp g2 = g;
        g2.active = g.active && ch.flag_rec;
        double f1[4];
        free_energy64(jb, tb64g, g2, vp, f1);
        loop_reduce4(f1, g2);
        Grp g3 = g2;
        g3.active = g2.active && ch.Fb != 0.0;
        double f2[4];
        free_energy64(jb, tb64g, g3, v, f2);
        loop_reduce4(f2, g3);
        // Kitaev: the FP64 eigen-stage of v' (and of v when its log-weight
        // came from the df64 stage), by the group that needs it
        double k1v[3] = {0.0, 0.0, 0.0}, k0v[3] = {0.0, 0.0, 0.0};
        const bool redo_v = ch.lpb != 0.0;
        if (KIND == kKitaev) {
          kitaev_logpi64<MULTI>(g, vp, jb.L, jb.J, ch.beta, wk, k1v, nullptr, jb.lc_edge > 0);
          if (redo_v) kitaev_logpi64<MULTI>(g, v, jb.L, jb.J, ch.beta, wk, k0v, nullptr, jb.lc_edge > 0);
        }
        if (g2.active && g.r == 0) {
          ch.Fp = -jb.vb * f1[2] - f1[0];
          ch.Bp = 0.0;
          if (g3.active) {
            ch.F = -jb.vb * f2[2] - f2[0];
            ch.Fb = 0.0;
          }
          if (KIND == kKitaev) {
            ch.lpp = k1v[0];
            ch.lppb = 0.0;
            ch.Ep = k1v[1];
            ch.otp[0] = k1v[1]; ch.otp[1] = k1v[1] * k1v[1]; ch.otp[2] = k1v[2];
            if (redo_v) {
              ch.lp = k0v[0];
              ch.lpb = 0.0;
            }
          }
          const double logr = (ch.lpp - ch.lp) + (ch.Fp - ch.F);
          const uint4 w = philox4x32_10_rk(make_uint4(0u, kTagAcc, step, g.cid), jb.rk);
          const double lu = log(((double)w.x + 0.5) * 0x1p-32);
          ch.flag_acc = lu < logr;
          if (KIND == kKitaev) ch.rec_mh += 1ull;   // Ising: counted at the df64 level
        }
      }
    }
    if (g.active && g.r == 0) {
      if (ch.flag_acc) {
        ch.cur ^= 1;
        ch.F = ch.Fp;
        ch.Fb = ch.Bp;
        ch.lp = ch.lpp;
        ch.lpb = ch.lppb;
        ch.E = ch.Ep;
        for (int o = 0; o < kNobs; ++o) ch.ot[o] = ch.otp[o];
        ch.acc += 1ull;
      }
      for (int o = 0; o < kNobs; ++o) ch.os[o] += ch.ot[o];
      trace_store(jb, g.c, step0 + (uint64_t)s, ch.E);
    }
    loop_sync();
  }

  if (nrec) atomicAdd(&ch.rec, (unsigned long long)nrec);
  __syncthreads();
  if (g.active) {
    const uint32_t* v = my + ch.cur * P;
    for (int w = g.r; w < jb.Wd; w += g.tpc) jb.bits[(size_t)g.c * jb.Wd + w] = v[w];
    if (g.r == 0) {
      jb.F[g.c] = ch.F;
      jb.Fb[g.c] = ch.Fb;
      jb.Lb[g.c] = ch.lpb;
      jb.logpi[g.c] = ch.lp;
      jb.Ephys[g.c] = ch.E;
      for (int o = 0; o < kNobs; ++o) {
        jb.obs_t[(size_t)g.c * kNobs + o] = ch.ot[o];
        jb.obs[(size_t)g.c * kNobs + o] = ch.os[o];
      }
      jb.acc[g.c] += ch.acc;
      jb.rec[2 * (size_t)g.c] += ch.rec;
      jb.rec[2 * (size_t)g.c + 1] += ch.rec_mh;
    }
  }
}


// After a launch of S proposals: every job's device step counter += S.
static __global__ void advance_steps_kernel(const __grid_constant__ LaunchParams p) {
  const int i = threadIdx.x;
  if (i < p.n_jobs) *p.job[i].step += (unsigned long long)p.S;
}

// Launch one instantiation; raise its dynamic shared-memory limit.  MULTI
// launches run mode 0 only.
template <int KIND, int PREC, int KC, int kC, int NT, bool MULTI = false>
cudaError_t launch_inst(const LaunchParams& p, int grid, size_t smem, cudaStream_t st) {
  if constexpr (MULTI) {
    crbm_step_kernel<KIND, PREC, KC, kC, NT, 0, true><<<grid, NT, smem, st>>>(p);
  } else {
    if (p.mode == 0) crbm_step_kernel<KIND, PREC, KC, kC, NT, 0><<<grid, NT, smem, st>>>(p);
    else crbm_step_kernel<KIND, PREC, KC, kC, NT, 1><<<grid, NT, smem, st>>>(p);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && p.mode != 1 && p.S > 0) {
    advance_steps_kernel<<<1, kMaxJobs, 0, st>>>(p);
    e = cudaGetLastError();
  }
  return e;
}

template <int KIND, int PREC, int KC, int kC, int NT>
cudaError_t limit_inst(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(crbm_step_kernel<KIND, PREC, KC, kC, NT, 0>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(crbm_step_kernel<KIND, PREC, KC, kC, NT, 1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

template <int KIND, int PREC, int NT>
cudaError_t launch_nt(int KC, int kC, const LaunchParams& p, int grid, size_t smem, cudaStream_t st) {
  if (KC == 4 && kC == 5) return launch_inst<KIND, PREC, 4, 5, NT>(p, grid, smem, st);
  if (KC == 4 && kC == 3) return launch_inst<KIND, PREC, 4, 3, NT>(p, grid, smem, st);
  return launch_inst<KIND, PREC, 0, 0, NT>(p, grid, smem, st);
}

template <int KIND, int PREC, int NT>
cudaError_t limit_nt(size_t bytes) {
  cudaError_t e = limit_inst<KIND, PREC, 4, 5, NT>(bytes);
  if (e == cudaSuccess) e = limit_inst<KIND, PREC, 4, 3, NT>(bytes);
  if (e == cudaSuccess) e = limit_inst<KIND, PREC, 0, 0, NT>(bytes);
  return e;
}

// The several-chains-per-CTA proposal kernel (mixed-size Kitaev batches).
template <int KIND, int PREC, int NT>
cudaError_t launch_multi(int KC, int kC, const LaunchParams& p, int grid, size_t smem, cudaStream_t st) {
  if (KC == 4 && kC == 5) return launch_inst<KIND, PREC, 4, 5, NT, true>(p, grid, smem, st);
  if (KC == 4 && kC == 3) return launch_inst<KIND, PREC, 4, 3, NT, true>(p, grid, smem, st);
  return launch_inst<KIND, PREC, 0, 0, NT, true>(p, grid, smem, st);
}

template <int KIND, int PREC, int NT>
cudaError_t limit_multi(size_t bytes) {
  cudaError_t e = cudaSuccess;
  for (auto f : {crbm_step_kernel<KIND, PREC, 4, 5, NT, 0, true>, crbm_step_kernel<KIND, PREC, 4, 3, NT, 0, true>,
                 crbm_step_kernel<KIND, PREC, 0, 0, NT, 0, true>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

// One translation unit per (kind, precision, CTA size) instantiates the
// (K, k) variants (4, 5), (4, 3) and runtime: CTAs of 256 threads, plus 128,
// 64 and 32 threads for the Kitaev kind (small matrices); every CTA size gets
// the same 128-register budget.  Separate units compile in parallel.
#define CRBM_VARIANTS_NT(KIND, PREC, NT)                                                       \
  cudaError_t launch_##KIND##_##PREC##_##NT(int KC, int kC, const LaunchParams& p, int grid,   \
                                            size_t smem, cudaStream_t st) {                    \
    return launch_nt<KIND, PREC, NT>(KC, kC, p, grid, smem, st);                               \
  }                                                                                            \
  cudaError_t limit_##KIND##_##PREC##_##NT(size_t bytes) { return limit_nt<KIND, PREC, NT>(bytes); }

#define CRBM_VARIANTS_MULTI(KIND, PREC, NT)                                                    \
  cudaError_t launch_##KIND##_##PREC##_##NT##_multi(int KC, int kC, const LaunchParams& p, int grid, \
                                                    size_t smem, cudaStream_t st) {            \
    return launch_multi<KIND, PREC, NT>(KC, kC, p, grid, smem, st);                            \
  }                                                                                            \
  cudaError_t limit_##KIND##_##PREC##_##NT##_multi(size_t bytes) { return limit_multi<KIND, PREC, NT>(bytes); }

}  // namespace crbm
