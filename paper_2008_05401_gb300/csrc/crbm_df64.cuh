// Double-FP32 ("df64") arithmetic and the Kitaev eigen-stage of the mixed path.
//
// A df64 value is an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, about 48 significant bits.  The error-free transforms are
// Knuth's TwoSum, Dekker's Fast2Sum and the FMA-based exact product; the
// add / mul / div / sqrt built from them follow Dekker (1971).  Each op
// carries a relative error below 2^-46, and every op costs a handful of FP32
// instructions -- on GB300, where FP64 runs at about 1/64 of the FP32 rate,
// that is several times cheaper than native FP64.
#pragma once
#include "crbm_device.cuh"

namespace crbm {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
// a + b with one normalisation (the reduction's sums of partials): TwoSum of
// the high parts, the low parts added in FP32; |error| <= 3 2^-48 (|a| + |b|)
// (no relative bound under cancellation).  Commutative, as df_add.
__device__ __forceinline__ df df_add_fast(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
// c + a b with one normalisation (the reduction's inner loops): a.hi b.hi
// exact by two_prod, its low part with the cross terms and c.lo in FP32, the
// high parts added by TwoSum.  Dropped a.lo b.lo and the FP32 roundings of
// the low sum give |error| <= 13 2^-48 |a b| + 3 2^-48 |c| < 2^-44 (|a b| +
// |c|) -- an absolute bound in the operands' size (no relative bound under
// cancellation), which is the form the backward-error analysis of the
// reduction uses (about 1.6 times the bound of df_mul then df_add).
__device__ __forceinline__ df df_fma(df a, df b, df c) {
  const df p = two_prod(a.hi, b.hi);
  const float t = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)) + c.lo;
  const df s = two_sum(c.hi, p.hi);
  return fast_two_sum(s.hi, s.lo + t);
}
// a - (x1 y1 + x2 y2) with one normalisation (the rank-2 update): the two
// high products exact, their low parts and the four cross terms summed in
// FP32, the high parts taken from a.hi by two TwoSums; |error| <= 2^-48
// (6 |a| + 21 |x1 y1| + 23 |x2 y2|) < 2^-43 (|a| + |x1 y1| + |x2 y2|), the
// same form as df_fma's (about 2.3 times the bound of two df_mul and two
// df_add).
__device__ __forceinline__ df df_sub_dot2(df a, df x1, df y1, df x2, df y2) {
  const df p1 = two_prod(x1.hi, y1.hi), p2 = two_prod(x2.hi, y2.hi);
  const float c = fmaf(x1.hi, y1.lo, fmaf(x1.lo, y1.hi, fmaf(x2.hi, y2.lo, fmaf(x2.lo, y2.hi, p1.lo + p2.lo))));
  const df s1 = two_sum(a.hi, -p1.hi);
  const df s2 = two_sum(s1.hi, -p2.hi);
  return fast_two_sum(s2.hi, ((a.lo - c) + s1.lo) + s2.lo);
}
// x1 y1 - x2 y2 with one normalisation (the Sturm recurrence): as
// df_sub_dot2 without a; |error| <= 2^-48 (15 |x1 y1| + 17 |x2 y2|), i.e.
// relative perturbations of the two products below 2^-43 each.
__device__ __forceinline__ df df_dot2m(df x1, df y1, df x2, df y2) {
  const df p1 = two_prod(x1.hi, y1.hi), p2 = two_prod(x2.hi, y2.hi);
  const float c = fmaf(x1.hi, y1.lo, fmaf(x1.lo, y1.hi, fmaf(-x2.hi, y2.lo, fmaf(-x2.lo, y2.hi, p1.lo - p2.lo))));
  const df s = two_sum(p1.hi, -p2.hi);
  return fast_two_sum(s.hi, s.lo + c);
}
__device__ __forceinline__ df df_div(df a, df b) {
  const float q1 = a.hi / b.hi;
  const df r = df_add(a, df_neg(df_mul(b, {q1, 0.0f})));
  const float q2 = r.hi / b.hi;
  const df r2 = df_add(r, df_neg(df_mul(b, {q2, 0.0f})));
  const float q3 = r2.hi / b.hi;
  const df q = fast_two_sum(q1, q2);
  return df_add(q, {q3, 0.0f});
}
__device__ __forceinline__ df df_sqrt(df a) {
  if (a.hi <= 0.0f) return {0.0f, 0.0f};
  const float y = sqrtf(a.hi);
  const df r = df_add(a, df_neg(two_prod(y, y)));   // a - y^2
  return fast_two_sum(y, r.hi / (2.0f * y));
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_from_float(float x) { return {x, 0.0f}; }

// ----------------------------------------------- double-FP32 softplus
// softplus(x) = max(x, 0) + log1p(e^-|x|) in df64, for the mixed path's
// second-level free energy (an MH decision that the FP32 bound cannot
// separate is retried with this one before the FP64 path's code runs).
// Table-driven exponential and logarithm in the manner of Tang (ACM TOMS 1989,
// 1990), with the leading terms kept exact by error-free transforms:
//   e^-a, 0 <= a <= 40: n = floor(a / ln2), s = a - n ln2 (n ln2.hi exact by
//     the FMA product, a.hi - n ln2.hi exact by Sterbenz; the low words in
//     FP32: |error| < 2.5 2^-42), m = rint(64 s) in [0, 44], r = s - m/64
//     (hi word exact, |r| <= 1/128 + 2^-25); e^-r = 1 - r + r^2/2 - r^3/6 +
//     r^4/24 - r^5/120 (remainder < 4e-16) with 1 - r.hi and r.hi^2 exact, the
//     terms beyond r^2 in FP32 (< 1e-7, error < 3e-14) and the low word of r
//     as - r.lo e^-r.hi; then e^-a = 2^-n e^(-m/64) e^-r with e^(-m/64) a df64
//     table entry (2^-48 relative) and one df64 product: relative error below
//     6.5e-13 in all;
//   log1p(e) = log u, u = 1 + e in [1, 2]: c = 1 + i/64 the nearest table
//     point, d = (u - c) / c with u - c exact (Sterbenz) and 1/c a df64 table
//     entry, |d| <= 2^-7; log u = log c + d - d^2/2 + d^3/3 - d^4/4 + d^5/5
//     (remainder < 4e-14), log c from the table, d - d.hi^2/2 exact, d.hi d.lo
//     and the terms beyond d^2 in FP32: absolute error below 2e-13 plus e's
//     relative error times e / (1 + e) <= 1/2;
//   a > 40: e^-a < 4.3e-18 and log1p(e) = e to within e^2, e from ex2.
// With the final df64 sum (2^-46 relative) the result is within
// 1e-12 + 2^-44 softplus(x) of the exact value (bound used by free_sum_df).
struct DfConst {
  float hi, lo;
};
constexpr DfConst dfc(double x) { return {(float)x, (float)(x - (double)(float)x)}; }
constexpr double exp_neg_m64(int m) {
  // e^(-m/64) by its Taylor series in double (host-side constant folding)
  double t = 1.0, s = 1.0, x = -(double)m / 64.0;
  for (int j = 1; j < 40; ++j) {
    t *= x / j;
    s += t;
  }
  return s;
}
constexpr double log_c64(int i) {
  // log(1 + i/64) = 2 atanh(z), z = i / (128 + i) <= 1/3: the odd series,
  // summed from its smallest term
  const double z = (double)i / (128.0 + (double)i), z2 = z * z;
  double t[40] = {};
  t[0] = z;
  for (int j = 1; j < 40; ++j) t[j] = t[j - 1] * z2;
  double s = 0.0;
  for (int j = 39; j >= 0; --j) s += t[j] / (double)(2 * j + 1);
  return 2.0 * s;
}
template <int N>
struct DfTable {
  DfConst v[N];
};
constexpr DfTable<45> make_exp_table() {
  DfTable<45> t{};
  for (int m = 0; m < 45; ++m) t.v[m] = dfc(exp_neg_m64(m));
  return t;
}
constexpr DfTable<65> make_log_table() {
  DfTable<65> t{};
  for (int i = 0; i < 65; ++i) t.v[i] = dfc(log_c64(i));
  return t;
}
constexpr DfTable<65> make_rcp_table() {
  DfTable<65> t{};
  for (int i = 0; i < 65; ++i) t.v[i] = dfc(64.0 / (64.0 + (double)i));
  return t;
}
// in global memory (L1-cached): the lanes of a warp index them at different
// points, which the constant cache would serve one address at a time
static __device__ const DfTable<45> kExpNegM64 = make_exp_table();   // e^(-m/64)
static __device__ const DfTable<65> kLogC64 = make_log_table();      // log(1 + i/64)
static __device__ const DfTable<65> kRcpC64 = make_rcp_table();      // 1 / (1 + i/64)

// e^-a for a df64 0 <= a <= 40.1.
__device__ __forceinline__ df df_exp_neg(df a) {
  constexpr DfConst ln2 = dfc(0.6931471805599453094172321);
  const float n = floorf(a.hi * 1.4426950408889634f);
  const df p = two_prod(n, ln2.hi);
  const df s = two_sum(a.hi - p.hi, fmaf(-n, ln2.lo, a.lo - p.lo));           // a - n ln2
  const float mf = fminf(fmaxf(rintf(s.hi * 64.0f), 0.0f), 44.0f);
  const float rh = s.hi - mf * 0.015625f, rl = s.lo;                          // r = s - m/64
  const df A = fast_two_sum(1.0f, -rh);
  const df q2 = two_prod(rh, rh);
  const df B = two_sum(A.hi, 0.5f * q2.hi);                                   // 1 - rh + rh^2/2
  const float R = rh * rh * rh * fmaf(rh, fmaf(rh, -1.0f / 120.0f, 1.0f / 24.0f), -1.0f / 6.0f);
  const float low = fmaf(-rl, B.hi, ((A.lo + B.lo) + 0.5f * q2.lo) + R);
  const df er = fast_two_sum(B.hi, low);                                      // e^-r
  const DfConst tm = kExpNegM64.v[(int)mf];
  const df t = df_mul(er, {tm.hi, tm.lo});
  const float sc = __int_as_float((127 - (int)n) << 23);     // 2^-n exactly (0 <= n <= 58)
  return {t.hi * sc, t.lo * sc};
}

// log(1 + e) for a df64 0 <= e <= 1.
__device__ __forceinline__ df df_log1p_unit(df e) {
  const df u0 = fast_two_sum(1.0f, e.hi);
  const float uh = u0.hi, ul = u0.lo + e.lo;                                  // u = 1 + e
  const int i = min(max(__float2int_rn((uh - 1.0f) * 64.0f), 0), 64);
  const float c = 1.0f + (float)i * 0.015625f;
  const DfConst rc = kRcpC64.v[i], lc = kLogC64.v[i];
  const df d = df_mul(two_sum(uh - c, ul), {rc.hi, rc.lo});                  // (u - c) / c
  const df s2 = two_prod(d.hi, d.hi);
  const df D = two_sum(d.hi, -0.5f * s2.hi);                                  // d.hi - d.hi^2/2
  const float C = d.hi * d.hi * d.hi * fmaf(d.hi, fmaf(d.hi, 0.2f, -0.25f), 1.0f / 3.0f);
  const df A = two_sum(lc.hi, D.hi);
  const float low = (((A.lo + D.lo) + (lc.lo + d.lo)) - fmaf(d.hi, d.lo, 0.5f * s2.lo)) + C;
  return fast_two_sum(A.hi, low);
}

// softplus(x) for a df64 x (see above).
__device__ __forceinline__ df softplus_df(df x) {
  const df a = x.hi < 0.0f ? df_neg(x) : x;
  const df pos = x.hi > 0.0f ? x : df{0.0f, 0.0f};
  if (a.hi > 40.0f) return df_add(pos, {ex2_approx(-a.hi * 1.4426950408889634f), 0.0f});
  return df_add(pos, df_log1p_unit(df_exp_neg(a)));
}

// Second-level free-energy sum of a lattice by a chain's group: the sum over
// units of softplus(h_bias + (W * v)), pre-activations from the hi/lo tables
// (hi sums exact in FP32, lo sums in FP32: within jb.cdf of the FP64 path's),
// softplus in df64.  out[0] = the group's partial sum, out[1] = a bound on its
// error against the FP64 path's terms, out[2] = ones of the lattice.
// KU: an upper bound on K known at compile time (the size of the register
// arrays; K <= KU).
template <int KU = kMaxK>
static __device__ __noinline__ void free_sum_df(const JobDev& jb, const Grp& g, const uint32_t* v, double* out) {
  const int L = jb.L, N = jb.N, K = jb.K, k = jb.k, T = 1 << k;
  df acc = {0.0f, 0.0f};
  float ssp = 0.0f;
  int units = 0, ones = 0;
  // one site per step; its k window codes index the tables as they are formed
  // (no per-thread code array, which would live in local memory) and the
  // pre-activations of its K hidden units stay in registers
  for (int n = g.active ? g.r : N; n < N; n += g.tpc) {
    const int i = n / L, j = n - i * L;
    ones += (int)((v[n >> 5] >> (n & 31)) & 1u);
    float xh[KU > 4 ? KU : 4], xl[KU > 4 ? KU : 4];
#pragma unroll
    for (int f = 0; f < (KU > 4 ? KU : 4); ++f) {
      xh[f] = f < K ? jb.hb_hi[f] : 0.0f;
      xl[f] = f < K ? jb.hb_lo[f] : 0.0f;
    }
    for (int a = 0; a < k; ++a) {
      const int r = i + a < L ? i + a : i + a - L;
      const int code = a * T + (int)row_window(v, L, r, j, k);
      if (K <= 4) {
        const float4 eh = __ldg(jb.fh4 + code), el = __ldg(jb.fl4 + code);
        xh[0] += eh.x; xh[1] += eh.y; xh[2] += eh.z; xh[3] += eh.w;
        xl[0] += el.x; xl[1] += el.y; xl[2] += el.z; xl[3] += el.w;
      } else {
#pragma unroll
        for (int f = 0; f < KU; ++f)
          if (f < K) {
            xh[f] += __ldg(jb.fh + f * k * T + code);
            xl[f] += __ldg(jb.fl + f * k * T + code);
          }
      }
    }
#pragma unroll
    for (int f = 0; f < KU; ++f)
      if (f < K) {
        const df sp = softplus_df(two_sum(xh[f], xl[f]));
        acc = df_add(acc, sp);
        ssp += sp.hi;
        ++units;
      }
  }
  out[0] = df_to_double(acc);
  // per unit 1e-12 + 2^-44 softplus (evaluation) + cdf (pre-activation);
  // the df64 running sum of <= 2^12 terms: 2^-34 of the sum of its terms
  out[1] = (double)units * (1e-12 + (double)jb.cdf) + (double)ssp * (0x1p-44 + 0x1p-34);
  out[2] = (double)ones;
}

// ----------------------------------------------- double-FP32 eigenvalue refinement
// The Sturm sequence p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} and its
// x-derivative in df64 arithmetic, for the mixed path's eigenvalues: the same
// FP32 bisection as the FP64 solver isolates eigenvalue idx, two df64 Sturm
// counts verify the padded bracket and safeguarded df64 Newton steps refine it
// -- on the FP32 pipe instead of GB300's slow FP64 one.  Values are kept
// between 2^-40 and 2^40 by exact power-of-two rescaling, so that the low
// words stay normal.  The computed counts are exact for a tridiagonal whose
// entries differ from (d, e^2) by a few units of 2^-46 relative (the
// backward stability of the Sturm recurrence, after Kahan), which moves
// every eigenvalue by at most 16 2^-46 (|d| + |e^2| scale); the log-weight
// bound of the mixed stage includes this.
__device__ __forceinline__ df df_of(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ df df_scale(df a, float s) { return {a.hi * s, a.lo * s}; }
__device__ __forceinline__ int df_expo(df a) { return (int)((__float_as_uint(a.hi) >> 23) & 0xffu); }

struct SturmNewtonDf {
  int cnt;
  df p, dp;
};

// Sign change count of the df64 Sturm sequence at x (with p_N and p_N').
template <bool DERIV>
__device__ inline SturmNewtonDf sturm_df(const df* d, const df* e2, int N, df x) {
  df pp = {1.0f, 0.0f}, p = df_add(d[0], df_neg(x));
  df dpp = {0.0f, 0.0f}, dp = {-1.0f, 0.0f};
  uint32_t sprev = 0u;
  uint32_t s = (p.hi == 0.0f) ? 1u : (__float_as_uint(p.hi) >> 31);
  int cnt = (int)(s ^ sprev);
  sprev = s;
  for (int i = 1; i < N; ++i) {
    const df dx = df_add(d[i], df_neg(x));
    const df pn = df_dot2m(dx, p, e2[i - 1], pp);
    if (DERIV) {
      const df dpn = df_sub_dot2(df_neg(p), df_neg(dx), dp, e2[i - 1], dpp);
      dpp = dp;
      dp = dpn;
    }
    pp = p;
    p = pn;
    s = (p.hi == 0.0f) ? (sprev ^ 1u) : (__float_as_uint(p.hi) >> 31);
    cnt += (int)(s ^ sprev);
    sprev = s;
    const int ex = DERIV ? max(df_expo(p), df_expo(dp)) : df_expo(p);
    if (ex > 127 + 40) {
      p = df_scale(p, 0x1p-40f);
      pp = df_scale(pp, 0x1p-40f);
      if (DERIV) {
        dp = df_scale(dp, 0x1p-40f);
        dpp = df_scale(dpp, 0x1p-40f);
      }
    } else if (ex < 127 - 40 && (DERIV ? max(df_expo(pp), df_expo(dpp)) : df_expo(pp)) < 127 - 40) {
      p = df_scale(p, 0x1p+40f);
      pp = df_scale(pp, 0x1p+40f);
      if (DERIV) {
        dp = df_scale(dp, 0x1p+40f);
        dpp = df_scale(dpp, 0x1p+40f);
      }
    }
  }
  return {cnt, p, dp};
}

// Eigenvalue idx (ascending) of the tridiagonal (d, e^2) in df64: FP32
// bisection (wk.d32 / wk.e32), df64 verification of the padded bracket
// (falling back to the Gershgorin interval), safeguarded df64 Newton.
__device__ inline double eigen_idx_df(const KitaevWork& wk, const EigGrid& gr, const df* d, const df* e2, int N,
                                      int idx, double glo, double ghi) {
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
  if (sturm_df<false>(d, e2, N, df_of(lo)).cnt > idx) lo = glo;
  if (sturm_df<false>(d, e2, N, df_of(hi)).cnt <= idx) hi = ghi;
  const double tol = 0x1p-42 * (range + fabs(glo));
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 100; ++it) {
    if (hi - lo <= tol) {
      x = 0.5 * (lo + hi);
      break;
    }
    const SturmNewtonDf r = sturm_df<true>(d, e2, N, df_of(x));
    if (r.cnt > idx) hi = x; else lo = x;
    const double step = df_to_double(df_div(r.p, r.dp));
    double xn = x - step;
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

// Sum of a df64 value over a warp (butterfly; df_add_fast is commutative, so
// every lane ends with the same value).
__device__ __forceinline__ df warp_sum_df(df x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df y = {__shfl_xor_sync(kFull, x.hi, o), __shfl_xor_sync(kFull, x.lo, o)};
    x = df_add_fast(x, y);
  }
  return x;
}

// Deterministic df64 sum over a chain's (warp-aligned) group, returned to
// every thread of it: warp sums, then the warps' partials in warp order.
// scratch: at least 32 doubles of the group.
template <bool MULTI>
__device__ __forceinline__ df grp_sum_df(df x, const Grp& g, double* scratch) {
  x = warp_sum_df(x);
  const int r = MULTI ? g.r : (int)threadIdx.x, tpc = MULTI ? g.tpc : (int)blockDim.x;
  const int warp = r >> 5, nw = tpc >> 5;
  df* sd = reinterpret_cast<df*>(scratch);
  grp_sync<MULTI>(g);
  if ((r & 31) == 0) sd[warp] = x;
  grp_sync<MULTI>(g);
  df s = sd[0];
  for (int w = 1; w < nw; ++w) s = df_add_fast(s, sd[w]);
  grp_sync<MULTI>(g);
  return s;
}

// Kitaev log-weight with the Householder tridiagonalisation of A = M^T M in
// df64 and the eigenvalues (FP32 isolation + FP64 Newton, as in the FP64
// stage) and sums in FP64.  res = {log pi, e, c_f, bound}: |log pi - exact| <=
// bound, from (i) the backward error of the reduction, taken as
// ||dA||_2 <= 8 N^2 2^-46 ||A||_F (Householder tridiagonalisation with unit
// roundoff 2^-46, constant 8 for safety), which by Weyl moves every
// eigenvalue mu = eps^2 by at most dmu, and (ii) the slope of
// log 2cosh(beta sqrt(mu)/2) in mu, at most min(beta^2/8, beta/(4 sqrt(mu))).
// Run by the chain's thread group g with its own work areas, like kitaev_logpi64.
template <bool MULTI>
__device__ inline void kitaev_logpi_df(const Grp& g, const uint32_t* v, int L, const double* J, double beta,
                                       const KitaevWork& wk, double (&res)[4], bool open_cols = false) {
  const int N = L * L, tid = MULTI ? g.r : (int)threadIdx.x, nt = MULTI ? g.tpc : (int)blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  df* A = reinterpret_cast<df*>(wk.A);        // same footprint as the FP64 matrix
  df* pw = reinterpret_cast<df*>(wk.pw);       // p, then w
  df* uu = reinterpret_cast<df*>(wk.vv);       // Householder vector u
  auto split = [](double x) -> df {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
  };
  const df tx = split(2.0 * J[0]), ty = split(2.0 * J[1]), tz = split(2.0 * J[2]);
  // A = M^T M, row w in the same fixed order as the FP64 stage (entries within
  // 2^-46 relative of the FP64 ones: part of the reduction's error budget)
  float fro = 0.0f;
  for (int w = tid; w < N; w += nt) {
    df* row = A + tri(w, 0);                    // lower-triangle row w: columns 0..w
    for (int c = 0; c <= w; ++c) row[c] = {0.0f, 0.0f};
    const int i = w / L, j = w - i * L;
    for (int typ = 0; typ < 3; ++typ) {
      int bi = i, bj = j;
      if (typ == 1) bi = (i == 0) ? L - 1 : i - 1;
      if (typ == 2) bj = (j == 0) ? L - 1 : j - 1;
      if (typ == 2 && open_cols && j == 0) continue;      // this y-bond crosses the open cut
      const int b = bi * L + bj;
      const df mz = site_bit(v, b) ? tz : df_neg(tz);
      const df mw = (typ == 0) ? mz : (typ == 1 ? tx : ty);
      const int wz = b;
      const int wx = ((bi + 1 == L) ? 0 : bi + 1) * L + bj;
      const int wy = bi * L + ((bj + 1 == L) ? 0 : bj + 1);
      if (wz <= w) row[wz] = df_add(row[wz], df_mul(mw, mz));
      if (wx <= w) row[wx] = df_add(row[wx], df_mul(mw, tx));
      if (wy <= w && !(open_cols && bj + 1 == L)) row[wy] = df_add(row[wy], df_mul(mw, ty));
    }
    for (int c = 0; c <= w; ++c) fro = fmaf((c == w ? 1.0f : 2.0f) * row[c].hi, row[c].hi, fro);
  }
  const double fro_all = grp_sum<MULTI>((double)fro, g, wk.sc);
  grp_sync<MULTI>(g);
  // Householder tridiagonalisation in df64, organised as the FP64 stage's
  // (kitaev_logpi64): u read from column j, three group barriers per column,
  // p = tau A22 u with H lanes per row, the rank-2 update element by element
  // over the packed triangle in folded order.  Every reduction stays in df64
  // on the FP32 pipe (an FP64 instruction costs tens of cycles of the SMSP's
  // FP64 pipe on GB300), the inner loops' multiply-adds, the update and the
  // sums with one normalisation each (df_fma, df_sub_dot2, df_add_fast).
  // sc[0..31]: per-warp df64 partials of p^T u, sc[32..63]: of s.
  df* scP = reinterpret_cast<df*>(wk.sc);
  df* scS = reinterpret_cast<df*>(wk.sc + 32);
  df s;
  {
    df s0 = {0.0f, 0.0f};
    for (int i = 2 + tid; i < N; i += nt) {
      const df a = A[tri(i, 0)];
      s0 = df_fma(a, a, s0);
    }
    s = grp_sum_df<MULTI>(s0, g, wk.sc);
  }
  for (int j = 0; j < N - 2; ++j) {
    const int m = N - j - 1, j1 = j + 1;
    const df x0 = A[tri(j1, j)];
    if (tid == 0) wk.d[j] = df_to_double(A[tri(j, j)]);
    if (s.hi == 0.0f) {
      // column already reduced: no reflection; s of the next column directly
      if (tid == 0) wk.e[j] = df_to_double(x0);
      df s2 = {0.0f, 0.0f};
      for (int i = j + 3 + tid; i < N; i += nt) {
        const df a = A[tri(i, j1)];
        s2 = df_fma(a, a, s2);
      }
      s = grp_sum_df<MULTI>(s2, g, wk.sc);
      continue;
    }
    const df nrm = df_sqrt(df_add(df_mul(x0, x0), s));
    const df alpha = (x0.hi >= 0.0f) ? df_neg(nrm) : nrm;
    const df u0 = df_add(x0, df_neg(alpha));
    const df tau = df_div({2.0f, 0.0f}, df_add(df_mul(u0, u0), s));
    if (tid == 0) wk.e[j] = df_to_double(alpha);
    // p_l = tau sum_c A22[l][c] u_c with H lanes per row, as in the FP64 stage
    const int H = row_split(m, nt), h = lane & (H - 1);
    df part = {0.0f, 0.0f};
    for (int l0 = 0; l0 < m; l0 += nt / H) {
      const int l = l0 + warp * (32 / H) + lane / H;
      df e0 = {0.0f, 0.0f}, e1 = {0.0f, 0.0f};
      if (l < m) {
        const df* row = A + tri(j1 + l, j1);
        int c = h;
        if (c == 0) {
          e0 = df_mul(row[0], u0);
          c = H;
        }
        for (; c + H <= l; c += 2 * H) {
          e1 = df_fma(row[c], A[tri(j1 + c, j)], e1);
          e0 = df_fma(row[c + H], A[tri(j1 + c + H, j)], e0);
        }
        if (c <= l) {
          e1 = df_fma(row[c], A[tri(j1 + c, j)], e1);
          c += H;
        }
        for (; c + H < m; c += 2 * H) {
          const int b1 = tri(j1 + c, 0), b2 = tri(j1 + c + H, 0);
          e0 = df_fma(A[b1 + j1 + l], A[b1 + j], e0);
          e1 = df_fma(A[b2 + j1 + l], A[b2 + j], e1);
        }
        if (c < m) {
          const int b1 = tri(j1 + c, 0);
          e0 = df_fma(A[b1 + j1 + l], A[b1 + j], e0);
        }
      }
      df e = df_add_fast(e0, e1);
      for (int o = 1; o < H; o <<= 1)
        e = df_add_fast(e, {__shfl_xor_sync(kFull, e.hi, o), __shfl_xor_sync(kFull, e.lo, o)});
      if (l < m && h == 0) {
        const df p = df_mul(tau, e), ul = l == 0 ? u0 : A[tri(j1 + l, j)];
        pw[l] = p;
        uu[l] = ul;
        part = df_fma(p, ul, part);
      }
    }
    part = warp_sum_df(part);
    if (lane == 0) scP[warp] = part;
    grp_sync<MULTI>(g);
    df pv = scP[0];
    for (int w = 1; w < nw; ++w) pv = df_add_fast(pv, scP[w]);
    const df Kc = df_mul(df_mul({0.5f, 0.0f}, tau), pv);
    for (int l = tid; l < m; l += nt) pw[l] = df_fma(df_neg(Kc), uu[l], pw[l]);
    grp_sync<MULTI>(g);
    // A22 -= u w^T + w u^T (u in uu, w in pw): column 0 of A22 with the
    // partials of s, then the rest of the packed triangle, as in the FP64 stage
    df sp = {0.0f, 0.0f};
    for (int r = tid; r < m; r += nt) {
      df* a = A + tri(j1 + r, j1);
      const df x = df_sub_dot2(*a, uu[r], pw[0], pw[r], u0);
      *a = x;
      if (r >= 2) sp = df_fma(x, x, sp);
    }
    const int ntri = (m - 1) * m / 2;
    FoldWalk fw(m - 1, tid, nt);
    for (int q = tid; q < ntri; q += nt, fw.next()) {
      int r, c;
      fw.rc(r, c);
      df* a = A + tri(j1 + 1 + r, j1 + 1 + c);
      *a = df_sub_dot2(*a, uu[r + 1], pw[c + 1], pw[r + 1], uu[c + 1]);
    }
    sp = warp_sum_df(sp);
    if (lane == 0) scS[warp] = sp;
    grp_sync<MULTI>(g);
    s = scS[0];
    for (int w = 1; w < nw; ++w) s = df_add_fast(s, scS[w]);
  }
  if (tid == 0) {
    wk.d[N - 2] = df_to_double(A[tri(N - 2, N - 2)]);
    wk.d[N - 1] = df_to_double(A[tri(N - 1, N - 1)]);
    wk.e[N - 2] = df_to_double(A[tri(N - 1, N - 2)]);
    wk.e[N - 1] = 0.0;
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
  // the df64 matrix is no longer needed: vv/pw hold FP64 Sturm data again
  // the matrix is reduced: its storage now holds the df64 tridiagonal (d, e^2)
  df* ddf = reinterpret_cast<df*>(wk.A);
  df* edf = ddf + N;
  for (int i = tid; i < N; i += nt) {
    wk.vv[i] = wk.e[i] * wk.e[i];
    wk.d32[i] = (float)wk.d[i];
    wk.e32[i] = (float)(wk.e[i] * wk.e[i]);
    ddf[i] = df_of(wk.d[i]);
    edf[i] = df_of(wk.e[i] * wk.e[i]);
  }
  const double glo = wk.sc[0], ghi = wk.sc[1];
  grp_sync<MULTI>(g);
  const EigGrid gr = eig_grid(wk, N, glo, ghi, tid, nt);
  grp_sync<MULTI>(g);
  // reduction backward error of this stage (constant 32: 8 for safety times
  // about 4 for the one-normalisation df_fma / df_sub_dot2 / df_add_fast of the
  // reduction's loops and sums) and of the FP64 stage it stands in for (8), the FP64 eigenvalue
  // solver's own error on the FP64 path's tridiagonal,
  // and this stage's df64 solver (Sturm backward error and Newton tolerance)
  const double scale = ghi - glo + fabs(glo) + fabs(ghi);
  const double dmu = ((double)N * (double)N * (32.0 * 0x1p-46 + 8.0 * 0x1p-53) * sqrt(fro_all) +
                      4.0 * (double)N * 0x1p-52 * (ghi - glo + fabs(glo)) +
                      16.0 * 0x1p-46 * scale + 2.0 * 0x1p-42 * (ghi - glo + fabs(glo))) * 1.01;
  double lp = 0.0, en = 0.0, cf = 0.0, bd = 0.0;
  for (int idx = tid; idx < N; idx += nt) {
    const double mu = fmax(eigen_idx_df(wk, gr, ddf, edf, N, idx, glo, ghi), 0.0);
    thermal_add(sqrt(mu), beta, lp, en, cf);
    const double mlo = fmax(mu - dmu, 0.0);
    const double slope = (mlo > 0.0) ? fmin(0.125 * beta * beta, 0.25 * beta / sqrt(mlo)) : 0.125 * beta * beta;
    bd += slope * dmu;
  }
  res[0] = grp_sum<MULTI>(lp, g, wk.sc);
  res[1] = grp_sum<MULTI>(en, g, wk.sc);
  res[2] = grp_sum<MULTI>(cf, g, wk.sc);
  res[3] = grp_sum<MULTI>(bd, g, wk.sc) * 1.01 + 1e-12 * fabs(res[0]) + 1e-300;
}

}  // namespace crbm
