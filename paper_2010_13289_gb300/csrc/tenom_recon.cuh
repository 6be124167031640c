/* Scalar TENO-M reconstruction on the device (Sections 2-3 of arXiv 2010.13289).
 *
 * Input: K register values v[0..K-1] = f_{i-K/2+1} .. f_{i+K/2}; output the reconstructed
 * h(x_{i+1/2}).  Steps in the paper's order:
 *   candidates f_{k,i+1/2} (Table 1),
 *   indicators beta_{k,r}, beta_K (Eq. measureTENO, 2nd line), tau_K (Eq. taukTENO),
 *   gamma_k = (1 + tau_K/(beta_k + 1e-40))^6 (Eq. measureTENO, C = 1, q = 6),
 *   chi_k = gamma_k / sum gamma (Eq. normalize), delta_k = [chi_k >= C_T] (Eq. cut-off),
 *   C_T constant or adaptive (TENO8A, Eqs. shock_indicator, cut-off_adjust),
 *   nonsmooth candidates filtered by MP (Eqs. minmod222-value_monotonicity_preserving)
 *   or replaced by the fixed TVD5 flux (Eqs. high order TVD-TVDbeta) (Eq. mp_flux),
 *   assembly with constant weights w_k = d_k (Eq. reconstuction, Section 3.3).
 * The indicators use exact sum-of-squares forms over the differences D_t = v[t+1] - v[t]
 * (teno_coeffs.cuh); the TVD5 flux is evaluated in its division-free difference form.
 * FP64 is the scarce resource on GB300: the cutoff compares gamma_k with C_T * sum gamma
 * (same truth value as chi_k < C_T, no division), 1/(beta_k + eps) is a Newton-Raphson
 * reciprocal, and every comparison, min/max and minmod runs on the integer pipe
 * (tenom_fastmath.cuh).
 */
#pragma once
#include <cstdint>
#include "teno_coeffs.cuh"
#include "tenom_fastmath.cuh"

namespace tenom {

enum { LIM_MP = 0, LIM_TVD5 = 1, LIM_VA = 2 };
enum { CT_CONST = 0, CT_ADAPTIVE = 1 };
enum { CURV_M4 = 0, CURV_MM = 1 };
enum { W_TENOM = 0, W_TENO = 1 };
enum { ST_RHO = 1, ST_P = 2, ST_ROE = 4, ST_NONFINITE = 8 };

struct SchemeDev {
  int ct_mode;
  int mp_curv;
  int weights;
  int default_d;         /* d_k are the maximal-order weights (central formula applies) */
  int exact_decisions;   /* 1: decide the cutoff in FP64 only (no certified FP32 filter) */
  int pad_;
  double ct_const;
  double mp_alpha;
  double mp_beta_third;  /* mp_beta / 3 */
  double d[6];
};

__device__ __forceinline__ double dmin(double a, double b) { return imin(a, b); }
__device__ __forceinline__ double dmax(double a, double b) { return imax(a, b); }

/* minmod of two arguments (Eq. minmod222; zero if an argument is zero). */
__device__ __forceinline__ double minmod2(double x, double y) {
  if (ipos(x) && ipos(y)) return imin(x, y);
  if (ineg(x) && ineg(y)) return imax(x, y);
  return 0.0;
}

/* minmod of four arguments (Eq. minmod444). */
__device__ __forceinline__ double minmod4(double a, double b, double c, double d) {
  if (ipos(a) && ipos(b) && ipos(c) && ipos(d)) return imin(imin(a, b), imin(c, d));
  if (ineg(a) && ineg(b) && ineg(c) && ineg(d)) return imax(imax(a, b), imax(c, d));
  return 0.0;
}

/* median(x, y, z) = x + minmod(y - x, z - x) (Eq. median). */
__device__ __forceinline__ double median3(double x, double y, double z) { return x + minmod2(y - x, z - x); }

/* MP bounds f^{L,min}, f^{L,max} at x_{i+1/2} (Eq. value_min_max); c = index of f_i. */
template <int c>
__device__ __forceinline__ void mp_bounds(const double* v, const SchemeDev& S, double& fmin, double& fmax) {
  const double dm1 = v[c] - 2.0 * v[c - 1] + v[c - 2];   /* d_{i-1} (Eq. curvature) */
  const double d0 = v[c + 1] - 2.0 * v[c] + v[c - 1];    /* d_i */
  const double dp1 = v[c + 2] - 2.0 * v[c + 1] + v[c];   /* d_{i+1} */
  double dhp, dhm;
  if (S.mp_curv == CURV_M4) {                            /* Eq. maximal_curvature */
    dhp = minmod4(4.0 * d0 - dp1, 4.0 * dp1 - d0, d0, dp1);
    dhm = minmod4(4.0 * dm1 - d0, 4.0 * d0 - dm1, dm1, d0);
  } else {
    dhp = minmod2(d0, dp1);
    dhm = minmod2(dm1, d0);
  }
  const double fi = v[c], fip = v[c + 1], fim = v[c - 1];
  const double f_ul = fi + S.mp_alpha * (fi - fim);          /* Eq. upper_limiter */
  const double f_md = 0.5 * (fi + fip) - 0.5 * dhp;          /* Eq. median_value */
  const double f_lc = fi + 0.5 * (fi - fim) + S.mp_beta_third * dhm;  /* Eq. large_curvature */
  fmin = imax(imin(imin(fi, fip), f_md), imin(imin(fi, f_ul), f_lc));
  fmax = imin(imax(imax(fi, fip), f_md), imax(imax(fi, f_ul), f_lc));
}

/* TVD5 flux f_i + phi delta^-/2 in difference form: with D_m = f_m - f_{m-1} and
   B = (-2 D_{i-1} + 11 D_i + 24 D_{i+1} - 3 D_{i+2})/30, phi delta^- is
   max(0, min(2D_i, 2D_{i+1}, B)) for D_i > 0, min(0, max(...)) for D_i < 0, 0 for D_i = 0. */
template <int c>
__device__ __forceinline__ double tvd5_flux(const double* v) {
  const double Dm = v[c - 1] - v[c - 2], D0 = v[c] - v[c - 1], Dp = v[c + 1] - v[c], Dpp = v[c + 2] - v[c + 1];
  const double B = (-2.0 * Dm + 11.0 * D0 + 24.0 * Dp - 3.0 * Dpp) * (1.0 / 30.0);
  double pd = 0.0;
  if (ipos(D0)) pd = imax(0.0, imin(imin(2.0 * D0, 2.0 * Dp), B));
  else if (ineg(D0)) pd = imin(0.0, imax(imax(2.0 * D0, 2.0 * Dp), B));
  return v[c] + 0.5 * pd;
}

/* Van Albada flux (Eqs. van_Albada_limiter, slop_ratio, vAflux, kappa = 1/3). */
template <int c>
__device__ __forceinline__ double va_flux(const double* v) {
  const double dm = v[c] - v[c - 1], dp = v[c + 1] - v[c];
  const double den = dp * dp + dm * dm;
  const double phi = den > 0.0 ? 2.0 * dp * dm / den : 0.0;
  const double kap = 1.0 / 3.0;
  return v[c] + phi / 4.0 * ((1.0 - kap * phi) * dm + (1.0 + kap * phi) * dp);
}

/* Adaptive C_T of TENO8A (Section 2.4); returns C_T and [beta] in *e. */
template <int c>
__device__ __forceinline__ double adaptive_ct(const double* D, int* e) {
  const double xi = 1e-3, Cr = 0.23, a1 = 10.5, a2 = 3.5;
  const double eps = 0.9 * Cr / (1.0 - 0.9 * Cr) * xi * xi;
  double eh = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    /* eta_{i-1+q}: Delta f_{j+1/2} = D[c + j], Delta f_{j-1/2} = D[c + j - 1] with j = q - 1 */
    const double dfp = D[c + q - 1], dfm = D[c + q - 2];
    const double eta = (iabs(2.0 * dfp * dfm) + eps) * rcp_nr1(dfp * dfp + dfm * dfm + eps);
    eh = (q == 0) ? eta : imin(eh, eta);
  }
  const double m = 1.0 - imin(1.0, eh * (1.0 / Cr));
  const double om = 1.0 - m;
  const double g = om * om * om * om * (1.0 + 4.0 * m);
  const double beta = a1 - a2 * (1.0 - g);
  int ex = (int)floor(beta);
  ex = ex < 7 ? 7 : (ex > 10 ? 10 : ex);
  *e = ex;
  return ex == 7 ? 1e-7 : (ex == 8 ? 1e-8 : (ex == 9 ? 1e-9 : 1e-10));
}

/* Certified single-precision evaluation of the cutoff decisions delta_k (and of [beta] of
   TENO8A).  FP32 runs on the SM's wide FP32 pipe; GB300's FP64 pipe is the bottleneck.
   Every FP32 indicator is evaluated together with its absolute-value form (same form,
   |coefficients|, on |D|), which bounds its rounding error: for a form with n differences,
   |beta_fp32 - beta| <= (3n + 7) u beta_abs with u = 2^-24 (dot-product error analysis,
   including the conversion of D to FP32); C = 64 u doubles that.  The bounds are carried
   through tau, gamma_k = (1 + tau/beta_k)^6 (scaled by the largest gamma to stay in range)
   and the comparison gamma_k < C_T sum gamma.  A decision is returned only when the whole
   interval lies on one side; otherwise (and for out-of-range data or an indicator that may
   vanish, where epsilon = 1e-40 matters) the caller decides in FP64.  Certified decisions
   equal the exact-arithmetic decisions, hence those of the FP64 path except where that
   path is itself within its rounding of the threshold (an adaptive-precision predicate in
   the sense of Shewchuk's robust geometric predicates). */
template <int K>
__device__ __forceinline__ bool cutoff_filter(const double (&D)[K - 1], const SchemeDev& S, unsigned& bits, int& ex) {
  constexpr int c = K / 2 - 1;
  constexpr int nk = K - 2;
  const float u = 5.9604645e-8f;
  const float C = 64.f * u;
  float d[K - 1], a[K - 1];
  float dmax = 0.f;
#pragma unroll
  for (int t = 0; t < K - 1; ++t) {
    d[t] = __double2float_rn(D[t]);
    a[t] = fabsf(d[t]);
    dmax = fmaxf(dmax, a[t]);
  }
  if (!(dmax <= 1e15f) || (dmax > 0.f && dmax < 1e-15f)) return false;
  float b[nk], e[nk];
  b[0] = beta0<c - 1, false, float>(d);
  e[0] = beta0<c - 1, true, float>(a);
  b[1] = beta1<c, false, float>(d);
  e[1] = beta1<c, true, float>(a);
  b[2] = beta2<c - 2, false, float>(d);
  e[2] = beta2<c - 2, true, float>(a);
  b[3] = beta3<c, false, float>(d);
  e[3] = beta3<c, true, float>(a);
  float bK, eK;
  if constexpr (K == 8) {
    b[4] = beta4<c - 3, false, float>(d);
    e[4] = beta4<c - 3, true, float>(a);
    b[5] = beta5<c, false, float>(d);
    e[5] = beta5<c, true, float>(a);
    bK = betaK8<0, false, float>(d);
    eK = betaK8<0, true, float>(a);
  } else {
    bK = betaK6<0, false, float>(d);
    eK = betaK6<0, true, float>(a);
  }
  const float comb = (b[1] + b[2] + 4.f * b[0]) * (1.f / 6.f);
  const float tau = fabsf(bK - comb);
  const float dtau = C * (eK + (e[1] + e[2] + 4.f * e[0]) * (1.f / 6.f)) + 8.f * u * (bK + comb);
  const float tl = fmaxf(tau - dtau, 0.f), th = tau + dtau;
  float xl[nk], xh[nk], xm = 1.f;
#pragma unroll
  for (int k = 0; k < nk; ++k) {
    const float bl = b[k] - C * e[k], bh = (b[k] + C * e[k]) * (1.f + 2.f * u);
    if (bl < 1e-30f) {
      if (th != 0.f) return false;  /* beta_k may vanish: epsilon matters */
      xl[k] = 1.f;
      xh[k] = 1.f;
    } else {
      xl[k] = (1.f + (tl / bh) * (1.f - 3.f * u)) * (1.f - u);
      xh[k] = (1.f + (th / bl) * (1.f + 3.f * u)) * (1.f + u);
      if (!(xh[k] < 1e30f)) return false;
    }
    xm = fmaxf(xm, xh[k]);
  }
  const float rxm = 1.f / xm;
  float gl[nk], gh[nk], Sl = 0.f, Sh = 0.f;
#pragma unroll
  for (int k = 0; k < nk; ++k) {
    const float yl = xl[k] * rxm * (1.f - 3.f * u), yh = xh[k] * rxm * (1.f + 3.f * u);
    const float yl3 = yl * yl * yl, yh3 = yh * yh * yh;
    gl[k] = yl3 * yl3 * (1.f - 8.f * u);
    gh[k] = yh3 * yh3 * (1.f + 8.f * u);
    Sl += gl[k];
    Sh += gh[k];
  }
  Sl *= 1.f - 8.f * u;
  Sh *= 1.f + 8.f * u;
  double CT = S.ct_const;
  ex = 7;
  if (S.ct_mode == CT_ADAPTIVE) {
    const float xi = 1e-3f, Cr = 0.23f, a1 = 10.5f, a2 = 3.5f;
    const float eps = 0.9f * Cr / (1.f - 0.9f * Cr) * xi * xi;
    float eh = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float dfp = d[c + q - 1], dfm = d[c + q - 2];
      const float eta = (fabsf(2.f * dfp * dfm) + eps) / (dfp * dfp + dfm * dfm + eps);
      eh = (q == 0) ? eta : fminf(eh, eta);
    }
    const float m = 1.f - fminf(1.f, eh / Cr);
    const float om = 1.f - m;
    const float g = om * om * om * om * (1.f + 4.f * m);
    const float beta = a1 - a2 * (1.f - g);
    if (fabsf(beta - rintf(beta)) < 1e-3f) return false;
    int x = (int)floorf(beta);
    x = x < 7 ? 7 : (x > 10 ? 10 : x);
    ex = x;
    CT = x == 7 ? 1e-7 : (x == 8 ? 1e-8 : (x == 9 ? 1e-9 : 1e-10));
  }
  const float CTf = __double2float_rn(CT);
  const float thl = CTf * (1.f - 2.f * u) * Sl * (1.f - u), thh = CTf * (1.f + 2.f * u) * Sh * (1.f + u);
  unsigned bt = 0;
#pragma unroll
  for (int k = 0; k < nk; ++k) {
    if (gh[k] < thl) continue;            /* certainly chi_k < C_T: delta_k = 0 */
    if (gl[k] >= thh) bt |= 1u << k;      /* certainly chi_k >= C_T: delta_k = 1 */
    else return false;
  }
  bits = bt;
  return true;
}

/* One TENO-M reconstruction.  flag receives delta bits | ([beta]-7) << 6; st receives
   ST_NONFINITE when an indicator is not finite. */
template <int K, int LIM>
__device__ __forceinline__ double teno_m(const double (&v)[K], const SchemeDev& S, unsigned& flag, int& st) {
  constexpr int c = K / 2 - 1;  /* index of f_i */
  constexpr int nk = K - 2;
  double D[K - 1];
#pragma unroll
  for (int t = 0; t < K - 1; ++t) D[t] = v[t + 1] - v[t];
  double fk[nk];
  unsigned bits = 0;
  int ex = 7;
  if (S.exact_decisions || !cutoff_filter<K>(D, S, bits, ex)) {
  double bk[nk];
  bk[0] = beta0<c - 1>(D);
  bk[1] = beta1<c>(D);
  bk[2] = beta2<c - 2>(D);
  bk[3] = beta3<c>(D);
  double bK;
  if constexpr (K == 8) {
    bk[4] = beta4<c - 3>(D);
    bk[5] = beta5<c>(D);
    bK = betaK8<0>(D);
  } else {
    bK = betaK6<0>(D);
  }
  const double tau = iabs(bK - (bk[1] + bk[2] + 4.0 * bk[0]) * (1.0 / 6.0));
  double gk[nk], sum = 0.0;
#pragma unroll
  for (int k = 0; k < nk; ++k) {
    const double x = fma(tau, rcp_nr1(bk[k] + 1e-40), 1.0);
    const double x3 = x * x * x;
    gk[k] = x3 * x3;
    sum += gk[k];
  }
  double CT = S.ct_const;
  if (S.ct_mode == CT_ADAPTIVE) CT = adaptive_ct<c>(D, &ex);
  /* chi_k < C_T  <=>  gamma_k < C_T sum gamma (all positive: compared as bit patterns) */
  const double thr = CT * sum;
  bits = 0;
#pragma unroll
  for (int k = 0; k < nk; ++k) bits |= (ilt_nonneg(gk[k], thr) ? 0u : 1u) << k;
  if (dbits(sum) >= 0x7ff0000000000000ll) st |= ST_NONFINITE;
  }
  flag = bits | ((unsigned)((ex - 7) & 3) << 6);
  constexpr unsigned all = (1u << nk) - 1u;
  if (bits == all && S.default_d) {
    /* every candidate smooth: sum_k d_k f_k is the K-point central scheme */
    if constexpr (K == 8) return central8<c>(v);
    else return central6<c>(v);
  }
  fk[0] = cand0<c>(v);
  fk[1] = cand1<c>(v);
  fk[2] = cand2<c>(v);
  fk[3] = cand3<c>(v);
  if constexpr (K == 8) {
    fk[4] = cand4<c>(v);
    fk[5] = cand5<c>(v);
  }
  if (S.weights == W_TENO) {
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int k = 0; k < nk; ++k)
      if (bits >> k & 1u) { num += S.d[k] * fk[k]; den += S.d[k]; }
    return num / den;
  }
  if (bits != all) {
    if constexpr (LIM == LIM_MP) {
      double fmin, fmax;
      mp_bounds<c>(v, S, fmin, fmax);
#pragma unroll
      for (int k = 0; k < nk; ++k)
        if (!(bits >> k & 1u)) fk[k] = median3(fk[k], fmin, fmax);
    } else {
      const double fl = (LIM == LIM_TVD5) ? tvd5_flux<c>(v) : va_flux<c>(v);
#pragma unroll
      for (int k = 0; k < nk; ++k)
        if (!(bits >> k & 1u)) fk[k] = fl;
    }
  }
  double f = 0.0;
#pragma unroll
  for (int k = 0; k < nk; ++k) f += S.d[k] * fk[k];
  return f;
}

}  // namespace tenom
