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
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }
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

// Kitaev log-weight with the Householder tridiagonalisation of A = M^T M in
// df64 and the eigenvalues (FP32 isolation + FP64 Newton, as in the FP64
// stage) and sums in FP64.  res = {log pi, e, c_f, bound}: |log pi - exact| <=
// bound, from (i) the backward error of the reduction, taken as
// ||dA||_2 <= 8 N^2 2^-46 ||A||_F (Householder tridiagonalisation with unit
// roundoff 2^-46, constant 8 for safety), which by Weyl moves every
// eigenvalue mu = eps^2 by at most dmu, and (ii) the slope of
// log 2cosh(beta sqrt(mu)/2) in mu, at most min(beta^2/8, beta/(4 sqrt(mu))).
__device__ inline void kitaev_logpi_df(const uint32_t* v, int L, const double* J, double beta,
                                       const KitaevWork& wk, double (&res)[4], bool open_cols = false) {
  const int N = L * L, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  df* A = reinterpret_cast<df*>(wk.A);        // same footprint as the FP64 matrix
  df* dv = reinterpret_cast<df*>(wk.vv);       // Householder vector
  df* pw = reinterpret_cast<df*>(wk.pw);       // p, then w
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
  const double fro_all = block_sum((double)fro, wk.sc);
  __syncthreads();
  for (int j = 0; j < N - 2; ++j) {
    const int m = N - j - 1;
    df s = {0.0f, 0.0f};
    for (int i = j + 2 + tid; i < N; i += nt) {
      const df a = A[tri(i, j)];
      s = df_fma(a, a, s);
    }
    // block sum of df partials (through doubles: exact enough, 2^-53)
    const double sd = block_sum(df_to_double(s), wk.sc);
    const df x0 = A[tri(j + 1, j)];
    if (tid == 0) wk.d[j] = df_to_double(A[tri(j, j)]);
    if (sd == 0.0) {
      if (tid == 0) wk.e[j] = df_to_double(x0);
      __syncthreads();
      continue;
    }
    const float sh = (float)sd;
    const df ss = {sh, (float)(sd - (double)sh)};
    const df nrm = df_sqrt(df_add(df_mul(x0, x0), ss));
    const df alpha = (x0.hi >= 0.0f) ? df_neg(nrm) : nrm;
    const df v0 = df_add(x0, df_neg(alpha));
    const df tau = df_div({2.0f, 0.0f}, df_add(df_mul(v0, v0), ss));
    if (tid == 0) wk.e[j] = df_to_double(alpha);
    for (int l = tid; l < m; l += nt) dv[l] = (l == 0) ? v0 : A[tri(j + 1 + l, j)];
    __syncthreads();
    for (int l = warp; l < m; l += nw) {
      df acc = {0.0f, 0.0f};
      for (int c = lane; c < m; c += 32) {
        const int off = (c <= l) ? tri(j + 1 + l, j + 1 + c) : tri(j + 1 + c, j + 1 + l);
        acc = df_fma(A[off], dv[c], acc);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const df other = {__shfl_xor_sync(kFull, acc.hi, o), __shfl_xor_sync(kFull, acc.lo, o)};
        acc = df_add(acc, other);
      }
      if (lane == 0) pw[l] = df_mul(tau, acc);
    }
    __syncthreads();
    df pv = {0.0f, 0.0f};
    for (int l = tid; l < m; l += nt) pv = df_fma(pw[l], dv[l], pv);
    const double pvd = block_sum(df_to_double(pv), wk.sc);
    const float ph = (float)pvd;
    const df Kc = df_mul(df_mul({0.5f, 0.0f}, tau), {ph, (float)(pvd - (double)ph)});
    for (int l = tid; l < m; l += nt) pw[l] = df_add(pw[l], df_neg(df_mul(Kc, dv[l])));
    __syncthreads();
    for (int l = warp; l < m; l += nw) {
      df* row = A + tri(j + 1 + l, j + 1);
      const df vl = dv[l], wl = pw[l];
      for (int c = lane; c <= l; c += 32)
        row[c] = df_add(row[c], df_neg(df_add(df_mul(vl, pw[c]), df_mul(wl, dv[c]))));
    }
    __syncthreads();
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
  __syncthreads();
  // the df64 matrix is no longer needed: vv/pw hold FP64 Sturm data again
  for (int i = tid; i < N; i += nt) {
    wk.vv[i] = wk.e[i] * wk.e[i];
    wk.d32[i] = (float)wk.d[i];
    wk.e32[i] = (float)(wk.e[i] * wk.e[i]);
  }
  const double glo = wk.sc[0], ghi = wk.sc[1];
  __syncthreads();
  // reduction backward error of this stage and of the FP64 stage it stands in
  // for, plus the FP64 eigenvalue solver's own error on either tridiagonal
  const double dmu = (8.0 * (double)N * (double)N * (0x1p-46 + 0x1p-53) * sqrt(fro_all) +
                      4.0 * (double)N * 0x1p-52 * (ghi - glo + fabs(glo))) * 1.01;
  double lp = 0.0, en = 0.0, cf = 0.0, bd = 0.0;
  for (int idx = tid; idx < N; idx += nt) {
    const double mu = fmax(eigen_idx(wk, N, idx, glo, ghi), 0.0);
    thermal_add(sqrt(mu), beta, lp, en, cf);
    const double mlo = fmax(mu - dmu, 0.0);
    const double slope = (mlo > 0.0) ? fmin(0.125 * beta * beta, 0.25 * beta / sqrt(mlo)) : 0.125 * beta * beta;
    bd += slope * dmu;
  }
  res[0] = block_sum(lp, wk.sc);
  res[1] = block_sum(en, wk.sc);
  res[2] = block_sum(cf, wk.sc);
  res[3] = block_sum(bd, wk.sc) * 1.01 + 1e-12 * fabs(res[0]) + 1e-300;
}

}  // namespace crbm
