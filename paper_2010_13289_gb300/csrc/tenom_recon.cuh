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
  float ct_const_f;       /* ct_const rounded to FP32 (certified filter) */
  double ct_const;
  double mp_alpha;
  double mp_beta_third;  /* mp_beta / 3 */
  double d[6];
};

__device__ __forceinline__ double dmin(double a, double b) { return imin(a, b); }
__device__ __forceinline__ double dmax(double a, double b) { return imax(a, b); }

/* minmod of two arguments (Eq. minmod222; zero if an argument is zero); k receives which
   argument was taken (0: x, 1: y, -1: zero). */
__device__ __forceinline__ double minmod2(double x, double y, int& k) {
  k = -1;
  if (ipos(x) && ipos(y)) {
    k = ilt(y, x) ? 1 : 0;
    return k ? y : x;
  }
  if (ineg(x) && ineg(y)) {
    k = ilt(x, y) ? 1 : 0;
    return k ? y : x;
  }
  return 0.0;
}
__device__ __forceinline__ double minmod2(double x, double y) {
  int k;
  return minmod2(x, y, k);
}

/* minmod of four arguments (Eq. minmod444); k receives the argument taken (0..3, -1: zero). */
__device__ __forceinline__ double minmod4(double a, double b, double c, double d, int& k) {
  k = -1;
  if (ipos(a) && ipos(b) && ipos(c) && ipos(d)) {
    const int kab = ilt(b, a) ? 1 : 0, kcd = ilt(d, c) ? 3 : 2;
    const double ab = kab ? b : a, cd = (kcd == 3) ? d : c;
    const bool r = ilt(cd, ab);
    k = r ? kcd : kab;
    return r ? cd : ab;
  }
  if (ineg(a) && ineg(b) && ineg(c) && ineg(d)) {
    const int kab = ilt(a, b) ? 1 : 0, kcd = ilt(c, d) ? 3 : 2;
    const double ab = kab ? b : a, cd = (kcd == 3) ? d : c;
    const bool r = ilt(ab, cd);
    k = r ? kcd : kab;
    return r ? cd : ab;
  }
  return 0.0;
}

/* median(x, y, z) = x + minmod(y - x, z - x) (Eq. median); sel receives 0 (x kept),
   1 (y) or 2 (z) -- the argument whose value the minmod moved x to. */
__device__ __forceinline__ double median3(double x, double y, double z, int& sel) {
  int k;
  const double m = minmod2(y - x, z - x, k);
  sel = k + 1;
  return x + m;
}
__device__ __forceinline__ double median3(double x, double y, double z) {
  int sel;
  return median3(x, y, z, sel);
}

/* MP bounds f^{L,min}, f^{L,max} at x_{i+1/2} (Eq. value_min_max); c = index of f_i.
   code receives the selections: [0] of d^{M4}_{i+1/2} and [1] of d^{M4}_{i-1/2} (the minmod
   argument, -1 zero; the 2-argument curvature maps d_i / d_{i+1} to 2 / 3), [2] of f^min
   and [3] of f^max (0 f_i, 1 f_{i+1}, 2 f^MD, 3 f^UL, 4 f^LC). */
template <int c>
__device__ __forceinline__ void mp_bounds(const double* v, const SchemeDev& S, double& fmin, double& fmax,
                                          int (&code)[4]) {
  const double dm1 = v[c] - 2.0 * v[c - 1] + v[c - 2];   /* d_{i-1} (Eq. curvature) */
  const double d0 = v[c + 1] - 2.0 * v[c] + v[c - 1];    /* d_i */
  const double dp1 = v[c + 2] - 2.0 * v[c + 1] + v[c];   /* d_{i+1} */
  double dhp, dhm;
  if (S.mp_curv == CURV_M4) {                            /* Eq. maximal_curvature */
    dhp = minmod4(4.0 * d0 - dp1, 4.0 * dp1 - d0, d0, dp1, code[0]);
    dhm = minmod4(4.0 * dm1 - d0, 4.0 * d0 - dm1, dm1, d0, code[1]);
  } else {
    int k0, k1;
    dhp = minmod2(d0, dp1, k0);
    dhm = minmod2(dm1, d0, k1);
    code[0] = k0 < 0 ? -1 : k0 + 2;
    code[1] = k1 < 0 ? -1 : k1 + 2;
  }
  const double fi = v[c], fip = v[c + 1], fim = v[c - 1];
  const double f_ul = fi + S.mp_alpha * (fi - fim);          /* Eq. upper_limiter */
  const double f_md = 0.5 * (fi + fip) - 0.5 * dhp;          /* Eq. median_value */
  const double f_lc = fi + 0.5 * (fi - fim) + S.mp_beta_third * dhm;  /* Eq. large_curvature */
  /* fmin = max(min(f_i, f_{i+1}, f^MD), min(f_i, f^UL, f^LC)); fmax mirrors it */
  {
    const int k1 = ilt(fip, fi) ? 1 : 0;
    const double t1 = k1 ? fip : fi;
    const int kL = ilt(f_md, t1) ? 2 : k1;
    const double L = (kL == 2) ? f_md : t1;
    const int k2 = ilt(f_ul, fi) ? 3 : 0;
    const double t2 = k2 ? f_ul : fi;
    const int kR = ilt(f_lc, t2) ? 4 : k2;
    const double R = (kR == 4) ? f_lc : t2;
    const bool r = ilt(L, R);
    fmin = r ? R : L;
    code[2] = r ? kR : kL;
  }
  {
    const int k1 = ilt(fi, fip) ? 1 : 0;
    const double t1 = k1 ? fip : fi;
    const int kL = ilt(t1, f_md) ? 2 : k1;
    const double L = (kL == 2) ? f_md : t1;
    const int k2 = ilt(fi, f_ul) ? 3 : 0;
    const double t2 = k2 ? f_ul : fi;
    const int kR = ilt(t2, f_lc) ? 4 : k2;
    const double R = (kR == 4) ? f_lc : t2;
    const bool r = ilt(R, L);
    fmax = r ? R : L;
    code[3] = r ? kR : kL;
  }
}
template <int c>
__device__ __forceinline__ void mp_bounds(const double* v, const SchemeDev& S, double& fmin, double& fmax) {
  int code[4];
  mp_bounds<c>(v, S, fmin, fmax, code);
}

/* TVD5 flux f_i + phi delta^-/2 in difference form: with D_m = f_m - f_{m-1} and
   B = (-2 D_{i-1} + 11 D_i + 24 D_{i+1} - 3 D_{i+2})/30, phi delta^- is
   max(0, min(2D_i, 2D_{i+1}, B)) for D_i > 0, min(0, max(...)) for D_i < 0, 0 for D_i = 0.
   pick receives the term taken: 0 (2D_i), 1 (2D_{i+1}), 2 (B), -1 (zero). */
template <int c>
__device__ __forceinline__ double tvd5_flux(const double* v, int& pick) {
  const double Dm = v[c - 1] - v[c - 2], D0 = v[c] - v[c - 1], Dp = v[c + 1] - v[c], Dpp = v[c + 2] - v[c + 1];
  const double B = (-2.0 * Dm + 11.0 * D0 + 24.0 * Dp - 3.0 * Dpp) * (1.0 / 30.0);
  double pd = 0.0;
  pick = -1;
  if (ipos(D0)) {
    int k = ilt(2.0 * Dp, 2.0 * D0) ? 1 : 0;
    double m = k ? 2.0 * Dp : 2.0 * D0;
    if (ilt(B, m)) { m = B; k = 2; }
    if (ilt(0.0, m)) { pd = m; pick = k; }
  } else if (ineg(D0)) {
    int k = ilt(2.0 * D0, 2.0 * Dp) ? 1 : 0;
    double m = k ? 2.0 * Dp : 2.0 * D0;
    if (ilt(m, B)) { m = B; k = 2; }
    if (ilt(m, 0.0)) { pd = m; pick = k; }
  }
  return v[c] + 0.5 * pd;
}
template <int c>
__device__ __forceinline__ double tvd5_flux(const double* v) {
  int pick;
  return tvd5_flux<c>(v, pick);
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
__device__ __forceinline__ double adaptive_ct(const double* D, int* e, double* beta_out = nullptr) {
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
  if (beta_out) *beta_out = beta;
  int ex = (int)floor(beta);
  ex = ex < 7 ? 7 : (ex > 10 ? 10 : ex);
  *e = ex;
  return ex == 7 ? 1e-7 : (ex == 8 ? 1e-8 : (ex == 9 ? 1e-9 : 1e-10));
}

/* Certified single-precision evaluation of the cutoff decisions delta_k (and of [beta] of
   TENO8A).  FP32 runs on the SM's wide FP32 pipe; GB300's FP64 pipe is the bottleneck.
   Every FP32 indicator is evaluated together with its absolute-value form (same form,
   |coefficients|, on |D|), which bounds its rounding error: for a form with n differences,
   |beta_fp32 - beta| <= (3n + 9) u beta_abs with u = 2^-24 (dot-product error analysis,
   including the conversion of D to FP32 by truncation, relative error below 2u; a
   difference below the FP32 normal range becomes 0, an absolute error far below the
   bound); C = 64 u covers n <= 7 with room.  The bounds are carried
   through tau, gamma_k = (1 + tau/beta_k)^6 (scaled by the largest gamma to stay in range)
   and the comparison gamma_k < C_T sum gamma (quotients by the fast division, whose 2-ulp
   error the bounds include).  A decision is returned only when the whole
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
    d[t] = f32_rz(D[t]);
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
      /* fast division: within 2 ulp (relative 4u) for divisors in [2^-126, 2^126] (here
         bl >= 1e-30 and, with |D| <= 1e15, bh < 1e33), hence 7u where a correctly rounded
         quotient needed 3u; an overflowing xh fails the range test below */
      xl[k] = (1.f + __fdividef(tl, bh) * (1.f - 7.f * u)) * (1.f - u);
      xh[k] = (1.f + __fdividef(th, bl) * (1.f + 7.f * u)) * (1.f + u);
      if (!(xh[k] < 1e30f)) return false;
    }
    xm = fmaxf(xm, xh[k]);
  }
  const float rxm = __fdividef(1.f, xm);  /* a common scale of every gamma: its rounding cancels */
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
  float CTf = S.ct_const_f;
  ex = 7;
  if (S.ct_mode == CT_ADAPTIVE) {
    const float xi = 1e-3f, Cr = 0.23f, a1 = 10.5f, a2 = 3.5f;
    const float eps = 0.9f * Cr / (1.f - 0.9f * Cr) * xi * xi;
    float eh = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float dfp = d[c + q - 1], dfm = d[c + q - 2];
      const float eta = __fdividef(fabsf(2.f * dfp * dfm) + eps, dfp * dfp + dfm * dfm + eps);
      eh = (q == 0) ? eta : fminf(eh, eta);
    }
    const float m = 1.f - fminf(1.f, eh * (1.f / Cr));
    const float om = 1.f - m;
    const float g = om * om * om * om * (1.f + 4.f * m);
    const float beta = a1 - a2 * (1.f - g);
    if (fabsf(beta - rintf(beta)) < 1e-3f) return false;
    int x = (int)floorf(beta);
    x = x < 7 ? 7 : (x > 10 ? 10 : x);
    ex = x;
    CTf = x == 7 ? 1e-7f : (x == 8 ? 1e-8f : (x == 9 ? 1e-9f : 1e-10f));
  }
  if (!(CTf >= 1e-30f)) return false;  /* C_T below the FP32 normal range: decide in FP64 */
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

/* Upper bound of sqrt(x) for x >= 0 from the fast reciprocal square root (within 2 ulp):
   x rsqrt(x) is within 5u of sqrt(x); the factor 1 + 8u makes it an upper bound. */
__device__ __forceinline__ float sqrt_up(float x) {
  const float u = 5.9604645e-8f;
  return x > 0.f ? x * rsqrtf(x) * (1.f + 8.f * u) : 0.f;
}

/* All-smooth screen of one split side from FP32 differences d[t] of the characteristic
 * sequence, each known only to within an absolute error E (the projection done in FP32 on
 * FP32 copies of the point data; the caller bounds E).  Returns true only when every
 * candidate is certainly smooth (delta_k = 1 for every k, Eq. cut-off); otherwise the
 * caller decides in FP64.  The decisions are bounded as in cutoff_filter (intervals of
 * beta_k and tau carried through gamma_k and the comparison gamma_k >= C_T sum gamma),
 * with these indicator bounds: the FP32 value of each beta = sum_j w_j t_j^2 on the given
 * d is within C u beta_abs(|d|) <= C u k dmax^2 (k = beta_abs(1, .., 1), the form with
 * |coefficients| on a vector of ones), and the error of d moves beta by at most
 * 2 sqrt(beta(d) k) E + k E^2 (Cauchy-Schwarz on sum_j w_j 2 |t_j| sum_i |m_ji| E).
 * TENO8A's [beta] (Eq. cut-off_adjust) is bounded by interval arithmetic: each eta_j over
 * the box |Delta f| +- E (numerator and denominator bounded separately), the minimum,
 * then m, g(m) and beta, which are monotone in eta; when both ends share one integer part
 * the test uses that [beta]'s C_T, otherwise C_T = 1e-7, the largest 10^-[beta], which
 * certifies the decisions for every [beta] (need_ex, for the flag byte: not certain). */
template <int K>
__device__ __forceinline__ bool screen_smooth(const float (&d)[K - 1], float E, const SchemeDev& S, bool need_ex,
                                              int& ex) {
  constexpr int c = K / 2 - 1;
  constexpr int nk = K - 2;
  const float u = 5.9604645e-8f;
  const float C = 64.f * u;
  float one[K - 1];
  float dmax = 0.f;
#pragma unroll
  for (int t = 0; t < K - 1; ++t) {
    one[t] = 1.f;
    dmax = fmaxf(dmax, fabsf(d[t]));
  }
  if (!(dmax <= 1e15f) || !(E <= 1e14f)) return false;
  const float dm2 = dmax * dmax;
  float b[nk], kk[nk];
  b[0] = beta0<c - 1, false, float>(d);
  kk[0] = beta0<c - 1, true, float>(one);
  b[1] = beta1<c, false, float>(d);
  kk[1] = beta1<c, true, float>(one);
  b[2] = beta2<c - 2, false, float>(d);
  kk[2] = beta2<c - 2, true, float>(one);
  b[3] = beta3<c, false, float>(d);
  kk[3] = beta3<c, true, float>(one);
  float bK, kK;
  if constexpr (K == 8) {
    b[4] = beta4<c - 3, false, float>(d);
    kk[4] = beta4<c - 3, true, float>(one);
    b[5] = beta5<c, false, float>(d);
    kk[5] = beta5<c, true, float>(one);
    bK = betaK8<0, false, float>(d);
    kK = betaK8<0, true, float>(one);
  } else {
    bK = betaK6<0, false, float>(d);
    kK = betaK6<0, true, float>(one);
  }
  auto err_of = [&](float bb, float kkb) {
    const float r = kkb * (C * dm2);
    return (r + kkb * E * E + 2.f * E * sqrt_up(kkb * (bb + r))) * (1.f + 16.f * u);
  };
  float er[nk];
#pragma unroll
  for (int k = 0; k < nk; ++k) er[k] = err_of(b[k], kk[k]);
  const float comb = (b[1] + b[2] + 4.f * b[0]) * (1.f / 6.f);
  const float dtau = (err_of(bK, kK) + (er[1] + er[2] + 4.f * er[0]) * (1.f / 6.f)) * (1.f + 8.f * u) +
                     8.f * u * (bK + comb);
  const float tau = fabsf(bK - comb);
  const float tl = fmaxf(tau - dtau, 0.f), th = tau + dtau;
  float xl[nk], xh[nk], xm = 1.f;
#pragma unroll
  for (int k = 0; k < nk; ++k) {
    const float bl = b[k] - er[k], bh = (b[k] + er[k]) * (1.f + 2.f * u);
    if (!(bl >= 1e-30f)) return false;  /* beta_k not bounded away from zero: undecided */
    /* fast division within 2 ulp (4u): bl >= 1e-30, bh < 1e33 */
    xl[k] = (1.f + __fdividef(tl, bh) * (1.f - 7.f * u)) * (1.f - u);
    xh[k] = (1.f + __fdividef(th, bl) * (1.f + 7.f * u)) * (1.f + u);
    if (!(xh[k] < 1e30f)) return false;
    xm = fmaxf(xm, xh[k]);
  }
  const float rxm = __fdividef(1.f, xm);  /* a common scale of every gamma: its rounding cancels */
  float gl[nk], Sh = 0.f;
#pragma unroll
  for (int k = 0; k < nk; ++k) {
    const float yl = xl[k] * rxm * (1.f - 3.f * u), yh = xh[k] * rxm * (1.f + 3.f * u);
    const float yl3 = yl * yl * yl, yh3 = yh * yh * yh;
    gl[k] = yl3 * yl3 * (1.f - 8.f * u);
    Sh += yh3 * yh3 * (1.f + 8.f * u);
  }
  Sh *= 1.f + 8.f * u;
  float CTf = (S.ct_mode == CT_ADAPTIVE) ? 1e-7f : S.ct_const_f;
  ex = 7;
  if (S.ct_mode == CT_ADAPTIVE) {
    const float xi = 1e-3f, Cr = 0.23f, a1 = 10.5f, a2 = 3.5f;
    const float eps = 0.9f * Cr / (1.f - 0.9f * Cr) * xi * xi;
    const float epl = eps * (1.f - 4.f * u), eph = eps * (1.f + 4.f * u);
    float el = 1.f, eh = 1.f;  /* bounds of eta_{i+1/2}; eta <= 1 always */
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float ap = fabsf(d[c + q - 1]), am = fabsf(d[c + q - 2]);
      const float apl = fmaxf(ap - E, 0.f), aml = fmaxf(am - E, 0.f), aph = ap + E, amh = am + E;
      /* three roundings in each; 8u covers them and the rounding of the product itself */
      const float nl = (2.f * apl * aml + epl) * (1.f - 8.f * u), nh = (2.f * aph * amh + eph) * (1.f + 8.f * u);
      const float dl = (apl * apl + aml * aml + epl) * (1.f - 8.f * u),
                  dh = (aph * aph + amh * amh + eph) * (1.f + 8.f * u);
      el = fminf(el, __fdividef(nl, dh) * (1.f - 8.f * u));  /* fast division: 4u */
      eh = fminf(eh, __fdividef(nh, dl) * (1.f + 8.f * u));
    }
    /* m decreases with eta, g decreases with m, beta increases with g */
    const float rCr = 1.f / Cr;
    const float mlo = 1.f - fminf(1.f, eh * rCr), mhi = 1.f - fminf(1.f, el * rCr);
    const float olo = 1.f - mhi, ohi = 1.f - mlo;
    const float glo = olo * olo * olo * olo * (1.f + 4.f * mhi), ghi = ohi * ohi * ohi * ohi * (1.f + 4.f * mlo);
    const float blo = a1 - a2 * (1.f - glo) - 1e-5f, bhi = a1 - a2 * (1.f - ghi) + 1e-5f;
    int xlo = (int)floorf(blo), xhi = (int)floorf(bhi);
    xlo = xlo < 7 ? 7 : (xlo > 10 ? 10 : xlo);
    xhi = xhi < 7 ? 7 : (xhi > 10 ? 10 : xhi);
    if (xlo == xhi) {  /* [beta] certain: its C_T */
      ex = xlo;
      CTf = ex == 7 ? 1e-7f : (ex == 8 ? 1e-8f : (ex == 9 ? 1e-9f : 1e-10f));
    } else if (need_ex) {
      return false;    /* the flag byte needs [beta] */
    }                  /* else C_T = 1e-7 bounds every [beta]'s C_T */
  }
  if (!(CTf >= 1e-30f)) return false;
  const float thh = CTf * (1.f + 2.f * u) * Sh * (1.f + u);
#pragma unroll
  for (int k = 0; k < nk; ++k)
    if (!(gl[k] >= thh)) return false;  /* not certainly chi_k >= C_T */
  return true;
}

/* Candidate k's Table 1 coefficients on v (c = index of f_i), read off the generated
   candidate formulas applied to unit vectors (compile-time constants for a constant k). */
template <int K>
__device__ __forceinline__ void cand_coeffs(int k, double (&g)[K]) {
  constexpr int c = K / 2 - 1;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double e[K];
#pragma unroll
    for (int j = 0; j < K; ++j) e[j] = (j == i) ? 1.0 : 0.0;
    double x = 0.0;
    switch (k) {
      case 0: x = cand0<c>(e); break;
      case 1: x = cand1<c>(e); break;
      case 2: x = cand2<c>(e); break;
      case 3: x = cand3<c>(e); break;
      case 4: if constexpr (K == 8) x = cand4<c>(e); break;
      default: if constexpr (K == 8) x = cand5<c>(e); break;
    }
    g[i] = x;
  }
}

/* the K-point central scheme's coefficients (all candidates smooth, w_k = maximal-order d_k) */
template <int K>
__device__ __forceinline__ void central_weights(double* om) {
  constexpr int c = K / 2 - 1;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double e[K];
#pragma unroll
    for (int i = 0; i < K; ++i) e[i] = (i == q) ? 1.0 : 0.0;
    if constexpr (K == 8) om[q] = central8<c>(e);
    else om[q] = central6<c>(e);
  }
}

/* Gradient on v of the MP bound selected by `code` (mp_bounds), with the curvature
   selections dcode[0] (d^{M4}_{i+1/2} = p0 d_i + p1 d_{i+1}) and dcode[1]
   (d^{M4}_{i-1/2} = m0 d_{i-1} + m1 d_i). */
template <int K>
__device__ __forceinline__ void mp_bound_grad(int code, const int (&dcode)[4], const SchemeDev& S, double (&g)[K]) {
  constexpr int c = K / 2 - 1;
  auto first = [](int k) { return k == 0 ? 4.0 : (k == 1 ? -1.0 : (k == 2 ? 1.0 : 0.0)); };
  auto second = [](int k) { return k == 0 ? -1.0 : (k == 1 ? 4.0 : (k == 3 ? 1.0 : 0.0)); };
#pragma unroll
  for (int i = 0; i < K; ++i) g[i] = 0.0;
  if (code == 0) {
    g[c] = 1.0;
  } else if (code == 1) {
    g[c + 1] = 1.0;
  } else if (code == 2) {  /* f^MD = (f_i + f_{i+1})/2 - d^{M4}_{i+1/2}/2 */
    const double p0 = first(dcode[0]), p1 = second(dcode[0]);
    g[c - 1] = -0.5 * p0;
    g[c] = 0.5 + p0 - 0.5 * p1;
    g[c + 1] = 0.5 - 0.5 * p0 + p1;
    g[c + 2] = -0.5 * p1;
  } else if (code == 3) {  /* f^UL = f_i + alpha (f_i - f_{i-1}) */
    g[c - 1] = -S.mp_alpha;
    g[c] = 1.0 + S.mp_alpha;
  } else {                 /* f^LC = f_i + (f_i - f_{i-1})/2 + (beta/3) d^{M4}_{i-1/2} */
    const double b0 = S.mp_beta_third * first(dcode[1]), b1 = S.mp_beta_third * second(dcode[1]);
    g[c - 2] = b0;
    g[c - 1] = -0.5 - 2.0 * b0 + b1;
    g[c] = 1.5 + b0 - 2.0 * b1;
    g[c + 1] = b1;
  }
}

/* Gradient on v of the TVD5 flux with the term `pick` (tvd5_flux) frozen. */
template <int K>
__device__ __forceinline__ void tvd5_grad(int pick, double (&g)[K]) {
  constexpr int c = K / 2 - 1;
#pragma unroll
  for (int i = 0; i < K; ++i) g[i] = 0.0;
  g[c] = 1.0;
  if (pick == 0) {         /* + D_i */
    g[c - 1] = -1.0;
    g[c] = 2.0;
  } else if (pick == 1) {  /* + D_{i+1} */
    g[c] = 0.0;
    g[c + 1] = 1.0;
  } else if (pick == 2) {  /* + B/2 */
    g[c - 2] = 2.0 / 60.0;
    g[c - 1] = -13.0 / 60.0;
    g[c] = 1.0 - 13.0 / 60.0;
    g[c + 1] = 27.0 / 60.0;
    g[c + 2] = -3.0 / 60.0;
  }
}

/* Cutoff decisions (delta bits, and [beta] of TENO8A in ex) in FP64: indicators beta_k,
   beta_K, tau_K, gamma_k and the comparison gamma_k < C_T sum gamma.  st receives
   ST_NONFINITE when an indicator is not finite. */
template <int K>
__device__ __forceinline__ void teno_decide_fp64(const double (&v)[K], const SchemeDev& S, unsigned& bits, int& ex,
                                                 int& st) {
  constexpr int c = K / 2 - 1;
  constexpr int nk = K - 2;
  double D[K - 1];
#pragma unroll
  for (int t = 0; t < K - 1; ++t) D[t] = v[t + 1] - v[t];
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
  ex = 7;
  if (S.ct_mode == CT_ADAPTIVE) CT = adaptive_ct<c>(D, &ex);
  /* chi_k < C_T  <=>  gamma_k < C_T sum gamma (all positive: compared as bit patterns) */
  const double thr = CT * sum;
  bits = 0;
#pragma unroll
  for (int k = 0; k < nk; ++k) bits |= (ilt_nonneg(gk[k], thr) ? 0u : 1u) << k;
  if (dbits(sum) >= 0x7ff0000000000000ll) st |= ST_NONFINITE;
}

/* Certified single-precision decisions (cutoff_filter); false: undecided, take the FP64
   path (always, when the scheme asks for FP64 decisions). */
template <int K>
__device__ __forceinline__ bool teno_decide_fast(const double (&v)[K], const SchemeDev& S, unsigned& bits, int& ex) {
  if (S.exact_decisions) return false;
  double D[K - 1];
#pragma unroll
  for (int t = 0; t < K - 1; ++t) D[t] = v[t + 1] - v[t];
  return cutoff_filter<K>(D, S, bits, ex);
}

/* every candidate smooth with the maximal-order d_k: sum_k d_k f_k is the K-point central
   scheme (WT: its constant weights into om) */
template <int K, bool WT = false>
__device__ __forceinline__ double teno_central(const double (&v)[K], double* om = nullptr) {
  constexpr int c = K / 2 - 1;
  if constexpr (WT) central_weights<K>(om);
  if constexpr (K == 8) return central8<c>(v);
  else return central6<c>(v);
}

/* Reconstruction with the cutoff decisions `bits` taken: candidates (Table 1), MP or TVD5
   filtering of the nonsmooth ones (Eq. mp_flux), assembly with w_k = d_k (Eq.
   reconstuction; with W_TENO the classical renormalised weights).  WT: om also receives
   the frozen linear weights of this evaluation, fhat = sum_q om_q v_q with these cutoff
   flags and this call's limiter selections (MP or TVD5 only). */
template <int K, int LIM, bool WT = false>
__device__ __forceinline__ double teno_general(const double (&v)[K], const SchemeDev& S, unsigned bits,
                                               double* om = nullptr) {
  static_assert(!WT || LIM == LIM_MP || LIM == LIM_TVD5, "frozen weights: MP or TVD5");
  constexpr int c = K / 2 - 1;  /* index of f_i */
  constexpr int nk = K - 2;
  constexpr unsigned all = (1u << nk) - 1u;
  if (bits == all && S.default_d) return teno_central<K, WT>(v, om);
  double fk[nk];
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
    if constexpr (WT) {
      const double rden = 1.0 / den;
#pragma unroll
      for (int i = 0; i < K; ++i) om[i] = 0.0;
#pragma unroll
      for (int k = 0; k < nk; ++k) {
        double g[K];
        cand_coeffs<K>(k, g);
        const double wk = (bits >> k & 1u) ? S.d[k] * rden : 0.0;
#pragma unroll
        for (int i = 0; i < K; ++i) om[i] = fma(wk, g[i], om[i]);
      }
    }
    return num / den;
  }
  /* per candidate: 0 used as it is, 1 replaced by the first frozen linear form (MP: f^min;
     TVD5: the TVD5 flux), 2 by the second (MP: f^max) */
  int sel[nk];
#pragma unroll
  for (int k = 0; k < nk; ++k) sel[k] = 0;
  int code[4] = {-1, -1, -1, -1};
  int pick = -1;
  if (bits != all) {
    if constexpr (LIM == LIM_MP) {
      double fmin, fmax;
      mp_bounds<c>(v, S, fmin, fmax, code);
#pragma unroll
      for (int k = 0; k < nk; ++k)
        if (!(bits >> k & 1u)) fk[k] = median3(fk[k], fmin, fmax, sel[k]);
    } else {
      const double fl = (LIM == LIM_TVD5) ? tvd5_flux<c>(v, pick) : va_flux<c>(v);
#pragma unroll
      for (int k = 0; k < nk; ++k)
        if (!(bits >> k & 1u)) {
          fk[k] = fl;
          sel[k] = 1;
        }
    }
  }
  double f = 0.0;
#pragma unroll
  for (int k = 0; k < nk; ++k) f += S.d[k] * fk[k];
  if constexpr (WT) {
    /* om = sum over unchanged candidates of d_k c_k + D1 grad(form 1) + D2 grad(form 2) */
    double D1 = 0.0, D2 = 0.0;
#pragma unroll
    for (int i = 0; i < K; ++i) om[i] = 0.0;
#pragma unroll
    for (int k = 0; k < nk; ++k) {
      double g[K];
      cand_coeffs<K>(k, g);
      const double wk = (sel[k] == 0) ? S.d[k] : 0.0;
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (g[i] != 0.0) om[i] = fma(wk, g[i], om[i]);
      D1 += (sel[k] == 1) ? S.d[k] : 0.0;
      D2 += (sel[k] == 2) ? S.d[k] : 0.0;
    }
    if (D1 != 0.0 || D2 != 0.0) {
      double g1[K], g2[K];
      if constexpr (LIM == LIM_MP) {
        mp_bound_grad<K>(code[2], code, S, g1);
        mp_bound_grad<K>(code[3], code, S, g2);
      } else {
        tvd5_grad<K>(pick, g1);
#pragma unroll
        for (int i = 0; i < K; ++i) g2[i] = 0.0;
      }
#pragma unroll
      for (int i = 0; i < K; ++i) om[i] = fma(D1, g1[i], fma(D2, g2[i], om[i]));
    }
  }
  return f;
}

/* One TENO-M reconstruction: decisions (certified FP32 filter, FP64 where it cannot decide)
   then teno_general.  flag receives delta bits | ([beta]-7) << 6. */
template <int K, int LIM, bool WT = false>
__device__ __forceinline__ double teno_m(const double (&v)[K], const SchemeDev& S, unsigned& flag, int& st,
                                         double* om = nullptr) {
  unsigned bits = 0;
  int ex = 7;
  if (!teno_decide_fast<K>(v, S, bits, ex)) teno_decide_fp64<K>(v, S, bits, ex, st);
  flag = bits | ((unsigned)((ex - 7) & 3) << 6);
  return teno_general<K, LIM, WT>(v, S, bits, om);
}

}  // namespace tenom
