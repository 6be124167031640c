/* Frozen-branch linear form of one TENO-M reconstruction (Sections 2-3 with every branch
 * taken from the forward pass).
 *
 * TENO-M assembles the candidates with constant weights w_k = d_k (Section 3.3), so once the
 * cutoff flags delta_k and the limiter's selections are fixed, the reconstruction is a LINEAR
 * function of the K stencil values: fhat = sum_q omega_q v_q.  teno_m_weights() replays the
 * forward's decisions on the same values (same expressions, same integer-pipe comparisons)
 * and returns omega.  No derivative flows through beta, tau, gamma or chi. */
#pragma once
#include "tenom_recon.cuh"

namespace tenom {

/* a value with its gradient with respect to the K stencil values */
template <int K>
struct Lin {
  double v;
  double g[K];
};

template <int K>
__device__ __forceinline__ Lin<K> lin_unit(const double* v, int q) {
  Lin<K> r;
  r.v = v[q];
#pragma unroll
  for (int i = 0; i < K; ++i) r.g[i] = (i == q) ? 1.0 : 0.0;
  return r;
}
template <int K>
__device__ __forceinline__ Lin<K> lin_zero() {
  Lin<K> r;
  r.v = 0.0;
#pragma unroll
  for (int i = 0; i < K; ++i) r.g[i] = 0.0;
  return r;
}
/* a*x + b*y + c*z with value computed in the forward's evaluation order by the caller */
template <int K>
__device__ __forceinline__ void lin_comb(Lin<K>& r, double a, const Lin<K>& x, double b, const Lin<K>& y) {
#pragma unroll
  for (int i = 0; i < K; ++i) r.g[i] = a * x.g[i] + b * y.g[i];
}
template <int K>
__device__ __forceinline__ Lin<K> lin_sel(bool take_b, const Lin<K>& a, const Lin<K>& b) { return take_b ? b : a; }

template <int K>
__device__ __forceinline__ Lin<K> lmin(const Lin<K>& a, const Lin<K>& b) { return lin_sel(ilt(b.v, a.v), a, b); }
template <int K>
__device__ __forceinline__ Lin<K> lmax(const Lin<K>& a, const Lin<K>& b) { return lin_sel(ilt(a.v, b.v), a, b); }

template <int K>
__device__ __forceinline__ Lin<K> lminmod2(const Lin<K>& x, const Lin<K>& y) {
  if (ipos(x.v) && ipos(y.v)) return lmin(x, y);
  if (ineg(x.v) && ineg(y.v)) return lmax(x, y);
  return lin_zero<K>();
}
template <int K>
__device__ __forceinline__ Lin<K> lminmod4(const Lin<K>& a, const Lin<K>& b, const Lin<K>& c, const Lin<K>& d) {
  if (ipos(a.v) && ipos(b.v) && ipos(c.v) && ipos(d.v)) return lmin(lmin(a, b), lmin(c, d));
  if (ineg(a.v) && ineg(b.v) && ineg(c.v) && ineg(d.v)) return lmax(lmax(a, b), lmax(c, d));
  return lin_zero<K>();
}

/* d = v[c+o+1] - 2 v[c+o] + v[c+o-1] */
template <int K>
__device__ __forceinline__ Lin<K> lin_curv(const double* v, int m) {
  Lin<K> r;
  r.v = v[m + 1] - 2.0 * v[m] + v[m - 1];
#pragma unroll
  for (int i = 0; i < K; ++i) r.g[i] = (i == m + 1 ? 1.0 : 0.0) - (i == m ? 2.0 : 0.0) + (i == m - 1 ? 1.0 : 0.0);
  return r;
}

/* gradient of the MP bounds (Eq. value_min_max) with the forward's selections */
template <int K, int c>
__device__ __forceinline__ void mp_bounds_lin(const double* v, const SchemeDev& S, Lin<K>& fmin, Lin<K>& fmax) {
  const Lin<K> dm1 = lin_curv<K>(v, c - 1), d0 = lin_curv<K>(v, c), dp1 = lin_curv<K>(v, c + 1);
  Lin<K> dhp, dhm;
  if (S.mp_curv == CURV_M4) {
    Lin<K> a1, a2, a3, a4;
    a1.v = 4.0 * d0.v - dp1.v;
    lin_comb(a1, 4.0, d0, -1.0, dp1);
    a2.v = 4.0 * dp1.v - d0.v;
    lin_comb(a2, 4.0, dp1, -1.0, d0);
    dhp = lminmod4(a1, a2, d0, dp1);
    a3.v = 4.0 * dm1.v - d0.v;
    lin_comb(a3, 4.0, dm1, -1.0, d0);
    a4.v = 4.0 * d0.v - dm1.v;
    lin_comb(a4, 4.0, d0, -1.0, dm1);
    dhm = lminmod4(a3, a4, dm1, d0);
  } else {
    dhp = lminmod2(d0, dp1);
    dhm = lminmod2(dm1, d0);
  }
  const Lin<K> fi = lin_unit<K>(v, c), fip = lin_unit<K>(v, c + 1), fim = lin_unit<K>(v, c - 1);
  Lin<K> f_ul, f_md, f_lc;
  f_ul.v = fi.v + S.mp_alpha * (fi.v - fim.v);
  lin_comb(f_ul, 1.0 + S.mp_alpha, fi, -S.mp_alpha, fim);
  f_md.v = 0.5 * (fi.v + fip.v) - 0.5 * dhp.v;
#pragma unroll
  for (int i = 0; i < K; ++i) f_md.g[i] = 0.5 * (fi.g[i] + fip.g[i]) - 0.5 * dhp.g[i];
  f_lc.v = fi.v + 0.5 * (fi.v - fim.v) + S.mp_beta_third * dhm.v;
#pragma unroll
  for (int i = 0; i < K; ++i) f_lc.g[i] = 1.5 * fi.g[i] - 0.5 * fim.g[i] + S.mp_beta_third * dhm.g[i];
  fmin = lmax(lmin(lmin(fi, fip), f_md), lmin(lmin(fi, f_ul), f_lc));
  fmax = lmin(lmax(lmax(fi, fip), f_md), lmax(lmax(fi, f_ul), f_lc));
}

/* gradient of the TVD5 flux in its difference form with the forward's selection */
template <int K, int c>
__device__ __forceinline__ void tvd5_lin(const double* v, double* g) {
  const double Dm = v[c - 1] - v[c - 2], D0 = v[c] - v[c - 1], Dp = v[c + 1] - v[c], Dpp = v[c + 2] - v[c + 1];
  const double B = (-2.0 * Dm + 11.0 * D0 + 24.0 * Dp - 3.0 * Dpp) * (1.0 / 30.0);
  /* coefficient vectors of 2 D_i, 2 D_{i+1}, B on v[c-2..c+2] */
  const double cD0[5] = {0.0, -2.0, 2.0, 0.0, 0.0};
  const double cDp[5] = {0.0, 0.0, -2.0, 2.0, 0.0};
  const double cB[5] = {2.0 / 30.0, (-2.0 - 11.0) / 30.0, (11.0 - 24.0) / 30.0, (24.0 + 3.0) / 30.0, -3.0 / 30.0};
  int pick = -1;  /* -1: zero, 0: 2D_i, 1: 2D_{i+1}, 2: B */
  if (ipos(D0)) {
    double m = 2.0 * D0;
    int k = 0;
    if (ilt(2.0 * Dp, m)) { m = 2.0 * Dp; k = 1; }
    if (ilt(B, m)) { m = B; k = 2; }
    pick = ilt(0.0, m) ? k : -1;  /* max(0, m): m wins only if 0 < m */
  } else if (ineg(D0)) {
    double m = 2.0 * D0;
    int k = 0;
    if (ilt(m, 2.0 * Dp)) { m = 2.0 * Dp; k = 1; }
    if (ilt(m, B)) { m = B; k = 2; }
    pick = ilt(m, 0.0) ? k : -1;  /* min(0, m) */
  }
#pragma unroll
  for (int i = 0; i < K; ++i) g[i] = (i == c) ? 1.0 : 0.0;
  if (pick >= 0) {
    const double* cc = pick == 0 ? cD0 : (pick == 1 ? cDp : cB);
#pragma unroll
    for (int t = 0; t < 5; ++t) g[c - 2 + t] += 0.5 * cc[t];
  }
}

/* Returns true when omega is exactly the central scheme (every candidate used as it is:
   smooth, or nonsmooth but left unchanged by the MP median) with the maximal-order d_k. */
template <int K, int LIM>
__device__ __forceinline__ bool teno_m_weights(const double (&v)[K], unsigned bits, const SchemeDev& S,
                                               double (&om)[K]) {
  constexpr int c = K / 2 - 1;
  constexpr int nk = K - 2;
#pragma unroll
  for (int i = 0; i < K; ++i) om[i] = 0.0;
  if (S.weights == W_TENO) {
    if (bits == (1u << nk) - 1u && S.default_d) {
      central_weights<K>(om);
      return true;
    }
    double den = 0.0;
#pragma unroll
    for (int k = 0; k < nk; ++k)
      if (bits >> k & 1u) den += S.d[k];
    const double rden = 1.0 / den;
#pragma unroll
    for (int k = 0; k < nk; ++k)
      if (bits >> k & 1u) {
        double g[K];
        cand_coeffs<K>(k, g);
#pragma unroll
        for (int i = 0; i < K; ++i) om[i] += S.d[k] * rden * g[i];
      }
    return false;
  }
  const bool all = bits == (1u << nk) - 1u;
  if (all && S.default_d) {  /* sum_k d_k f_k = the central scheme: constant weights */
    central_weights<K>(om);
    return true;
  }
  bool changed = false;  /* a limiter replaced some candidate */
  Lin<K> fmin, fmax;
  double gt[K];
  if (!all) {
    if constexpr (LIM == LIM_MP) mp_bounds_lin<K, c>(v, S, fmin, fmax);
    else tvd5_lin<K, c>(v, gt);
  }
#pragma unroll
  for (int k = 0; k < nk; ++k) {
    double g[K];
    if ((bits >> k & 1u) || LIM == LIM_MP) cand_coeffs<K>(k, g);
    if (!(bits >> k & 1u)) {
      if constexpr (LIM == LIM_MP) {
        /* median(f, fmin, fmax) = f + minmod(fmin - f, fmax - f): selects f, fmin or fmax */
        double fk = 0.0;
        switch (k) {
          case 0: fk = cand0<c>(v); break;
          case 1: fk = cand1<c>(v); break;
          case 2: fk = cand2<c>(v); break;
          case 3: fk = cand3<c>(v); break;
          case 4: if constexpr (K == 8) fk = cand4<c>(v); break;
          default: if constexpr (K == 8) fk = cand5<c>(v); break;
        }
        const double x = fmin.v - fk, y = fmax.v - fk;
        if (ipos(x) && ipos(y)) {
          const bool ymin = ilt(y, x);
          changed = true;
#pragma unroll
          for (int i = 0; i < K; ++i) g[i] = ymin ? fmax.g[i] : fmin.g[i];
        } else if (ineg(x) && ineg(y)) {
          const bool ymax = ilt(x, y);
          changed = true;
#pragma unroll
          for (int i = 0; i < K; ++i) g[i] = ymax ? fmax.g[i] : fmin.g[i];
        }
      } else {
        changed = true;
#pragma unroll
        for (int i = 0; i < K; ++i) g[i] = gt[i];
      }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) om[i] += S.d[k] * g[i];
  }
  if (!changed && S.default_d) {
    central_weights<K>(om);
    return true;
  }
  return false;
}

template <int K>
__device__ __forceinline__ double central_fn(const double* v) {
  if constexpr (K == 8) return central8<K / 2 - 1>(v);
  else return central6<K / 2 - 1>(v);
}

}  // namespace tenom
