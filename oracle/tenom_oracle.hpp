/* TENO-M CPU oracle: plain, slow, FP64 restatement of the method of
   Li, Fu & Adams, "A low-dissipation shock-capturing framework with flexible
   nonlinear dissipation control" (arXiv 2010.13289).

   TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
   CPU-baseline leg may load this code.  It shares nothing with the CUDA path.

   Every routine is templated on the scalar type T so that the same source runs with
     - double          (the oracle proper),
     - orc::Dual       (forward-mode derivative; every branch decided on the real part,
                        i.e. the frozen-branch linearisation used to check the adjoint),
     - orc::Counted    (counts FP64 operations: the algorithmic flop figure).

   Readings of points the paper leaves open are marked "reading:" where used.
   The positivity-preserving flux limiter (Section 4.4) is pinned by
   tests/test_oracle_positivity.py (segment and floor properties, exactness where it is
   inactive, conservation, Le Blanc against the exact Riemann solution).
   Parity-unpinned parts (no printed example exists): the adaptive cutoff C_T of
   TENO8A (Eqs. shock_indicator, cut-off_adjust) beyond its printed constants. */
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>
#include "beta_forms.h"

namespace orc {

/* ------------------------------------------------------------------ scalar types */
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual sqrt_(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.v > 0 ? a.d / (2.0 * s) : 0.0);
}
inline double val(const Dual& a) { return a.v; }

extern thread_local long long g_flops;  /* op counter for Counted */
struct Counted {
  double v;
  Counted() : v(0) {}
  Counted(double x) : v(x) {}
};
inline Counted operator+(Counted a, Counted b) { ++g_flops; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { ++g_flops; return Counted(a.v - b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline Counted operator*(Counted a, Counted b) { ++g_flops; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { ++g_flops; return Counted(a.v / b.v); }
inline Counted sqrt_(Counted a) { ++g_flops; return Counted(std::sqrt(a.v)); }
inline double val(const Counted& a) { return a.v; }
inline void count_cmp(const Counted&) { ++g_flops; }

inline double sqrt_(double a) { return std::sqrt(a); }
inline double val(double a) { return a; }
template <class T> inline void count_cmp(const T&) {}

/* Branches are decided on real parts; on equality the first argument wins
   (reading: tie-break rule, used identically for max/min/median/argmax). */
template <class T> inline bool lt(const T& a, const T& b) { count_cmp(a); return val(a) < val(b); }
template <class T> inline T max_(const T& a, const T& b) { return lt(a, b) ? b : a; }
template <class T> inline T min_(const T& a, const T& b) { return lt(b, a) ? b : a; }
template <class T> inline T abs_(const T& a) { count_cmp(a); return val(a) < 0 ? -a : a; }
template <class T> inline double sgn(const T& a) {
  count_cmp(a);
  double x = val(a);
  return x > 0 ? 1.0 : (x < 0 ? -1.0 : 0.0);  /* reading: sgn(0) = 0 */
}

/* ------------------------------------------------------------------ scheme */
enum { LIM_MP = 0, LIM_TVD5 = 1, LIM_VA = 2 };
enum { CT_CONST = 0, CT_ADAPTIVE = 1 };
enum { CURV_M4 = 0, CURV_MM = 1 };
enum { W_TENOM = 0, W_TENO = 1 };
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1 };

struct Scheme {
  int K;            /* 6 or 8 */
  int limiter;      /* LIM_* */
  int ct_mode;      /* CT_* */
  double ct_const;  /* C_T when ct_mode == CT_CONST */
  double mp_alpha;  /* alpha of Eq. upper_limiter (1.25) */
  double mp_beta;   /* beta of Eq. large_curvature (4) */
  int mp_curv;      /* d_{i+1/2}: M4 (Eq. maximal_curvature) or MM (minmod(d_i, d_{i+1})) */
  int weights;      /* W_TENOM: Eq. reconstuction with w_k = d_k (Section 3.3);
                       W_TENO: standard renormalised weights, Eq. weight_renormalize */
  double d[6];      /* optimal linear weights d_k */
  int positivity;   /* 1: positivity-preserving flux limiter in every RK stage (Section 4.4) */
};

/* Optimal linear weights.  The paper does not print them (Section 3.3 allows
   maximal-order or spectrally optimised d_k); reading: maximal order, i.e. the d_k for
   which sum_k d_k f_k reproduces the K-point central reconstruction.  Pinned by the
   order and linear-reproduction tests. */
inline void default_weights(int K, double* d) {
  if (K == 6) {
    d[0] = 9.0 / 20.0; d[1] = 6.0 / 20.0; d[2] = 1.0 / 20.0; d[3] = 4.0 / 20.0;
    d[4] = 0; d[5] = 0;
  } else {
    d[0] = 3.0 / 7.0; d[1] = 9.0 / 35.0; d[2] = 2.0 / 35.0; d[3] = 6.0 / 35.0;
    d[4] = 1.0 / 70.0; d[5] = 1.0 / 14.0;
  }
}

/* Diagnostics of one scalar reconstruction. */
struct ReconDiag {
  int delta_bits;      /* bit k = delta_k of Eq. cut-off */
  int ct_exp;          /* [beta] of Eq. cut-off_adjust (0 when C_T is constant) */
  double cut_rel[6];   /* (chi_k - C_T) / C_T : distance of chi_k from the cutoff */
  double beta_ct;      /* beta of Eq. cut-off_adjust (adaptive C_T), else 0 */
  int nonfinite;       /* gamma_k or chi_k not finite */
};

/* ------------------------------------------------------------------ Table 1 */
/* Candidate numerical fluxes f_{k,i+1/2} = sum_m c_m f_m (Section 3.1, Table 1).
   F(m) returns f_{i+m}. */
template <class T, class FN>
inline T candidate(int k, FN F) {
  switch (k) {
    case 0: return -1.0 / 6.0 * F(-1) + 5.0 / 6.0 * F(0) + 2.0 / 6.0 * F(1);
    case 1: return 2.0 / 6.0 * F(0) + 5.0 / 6.0 * F(1) - 1.0 / 6.0 * F(2);
    case 2: return 2.0 / 6.0 * F(-2) - 7.0 / 6.0 * F(-1) + 11.0 / 6.0 * F(0);
    case 3: return 3.0 / 12.0 * F(0) + 13.0 / 12.0 * F(1) - 5.0 / 12.0 * F(2) + 1.0 / 12.0 * F(3);
    case 4: return -3.0 / 12.0 * F(-3) + 13.0 / 12.0 * F(-2) - 23.0 / 12.0 * F(-1) + 25.0 / 12.0 * F(0);
    default: return 12.0 / 60.0 * F(0) + 77.0 / 60.0 * F(1) - 43.0 / 60.0 * F(2) + 17.0 / 60.0 * F(3)
                    - 3.0 / 60.0 * F(4);
  }
}

/* Smoothness indicator of the polynomial defined by a stencil (Section 2.2):
   beta = sum_{j=1}^{r-1} dx^{2j-1} int_{x_{i-1/2}}^{x_{i+1/2}} (d^j h/dx^j)^2 dx, with the
   Taylor coefficients a_l = sum_m M[l][m] (f_m - f_i) and the exact Gram matrix G of the
   derivative products (both from oracle/gen_beta.py). */
template <class T, class FN>
inline T beta_of(int r, int j0, const double* Mrows, const double* G, FN F) {
  T a[8];
  T fi = F(0);
  for (int l = 0; l < r - 1; ++l) {
    T s = 0.0;
    for (int m = 0; m < r; ++m) s = s + Mrows[l * r + m] * (F(j0 + m) - fi);
    a[l] = s;
  }
  T b = 0.0;
  for (int l = 0; l < r - 1; ++l)
    for (int lp = 0; lp < r - 1; ++lp) b = b + G[l * (r - 1) + lp] * (a[l] * a[lp]);
  return b;
}

template <class T, class FN>
inline T beta_candidate(int k, FN F) {
  switch (k) {
    case 0: return beta_of<T>(ORC_S0_R, ORC_S0_J0, &ORC_S0_M[0][0], &ORC_S0_G[0][0], F);
    case 1: return beta_of<T>(ORC_S1_R, ORC_S1_J0, &ORC_S1_M[0][0], &ORC_S1_G[0][0], F);
    case 2: return beta_of<T>(ORC_S2_R, ORC_S2_J0, &ORC_S2_M[0][0], &ORC_S2_G[0][0], F);
    case 3: return beta_of<T>(ORC_S3_R, ORC_S3_J0, &ORC_S3_M[0][0], &ORC_S3_G[0][0], F);
    case 4: return beta_of<T>(ORC_S4_R, ORC_S4_J0, &ORC_S4_M[0][0], &ORC_S4_G[0][0], F);
    default: return beta_of<T>(ORC_S5_R, ORC_S5_J0, &ORC_S5_M[0][0], &ORC_S5_G[0][0], F);
  }
}

/* beta_K on the K-point full stencil.  Reading: the same Jiang-Shu measure applied to
   the degree-(K-1) polynomial of the full stencil (Eq. taukTENO only names it). */
template <class T, class FN>
inline T beta_full(int K, FN F) {
  if (K == 6) return beta_of<T>(ORC_F6_R, ORC_F6_J0, &ORC_F6_M[0][0], &ORC_F6_G[0][0], F);
  return beta_of<T>(ORC_F8_R, ORC_F8_J0, &ORC_F8_M[0][0], &ORC_F8_G[0][0], F);
}

/* ------------------------------------------------------------------ limiters */
/* Eq. minmod222 */
template <class T> inline T minmod2(const T& x, const T& y) {
  return 0.5 * (sgn(x) + sgn(y)) * min_(abs_(x), abs_(y));
}
/* Eq. minmod444 */
template <class T> inline T minmod4(const T& a, const T& b, const T& c, const T& d) {
  double s = 0.125 * (sgn(a) + sgn(b)) * std::fabs((sgn(a) + sgn(c)) * (sgn(a) + sgn(d)));
  return s * min_(min_(abs_(a), abs_(b)), min_(abs_(c), abs_(d)));
}
/* Eq. median */
template <class T> inline T median(const T& x, const T& y, const T& z) { return x + minmod2(y - x, z - x); }
template <class T> inline T min3(const T& a, const T& b, const T& c) { return min_(min_(a, b), c); }
template <class T> inline T max3(const T& a, const T& b, const T& c) { return max_(max_(a, b), c); }

/* MP bounds (Section 3.2.2): f^{L,min}, f^{L,max} of Eq. value_min_max, from
   Eqs. curvature, maximal_curvature, upper_limiter, median_value, large_curvature.
   Reading: d^{MD}_{i+1/2} and d^{LC}_{i-1/2} both take the chosen curvature measure
   (M4 by default; MM = minmod(d_i, d_{i+1}), Section 4). */
template <class T, class FN>
inline void mp_bounds(const Scheme& S, FN F, T* fmin, T* fmax) {
  T dm1 = F(0) - 2.0 * F(-1) + F(-2);  /* d_{i-1} */
  T d0 = F(1) - 2.0 * F(0) + F(-1);    /* d_i */
  T dp1 = F(2) - 2.0 * F(1) + F(0);    /* d_{i+1} */
  T dhp, dhm;                          /* d_{i+1/2}, d_{i-1/2} */
  if (S.mp_curv == CURV_M4) {
    dhp = minmod4(4.0 * d0 - dp1, 4.0 * dp1 - d0, d0, dp1);
    dhm = minmod4(4.0 * dm1 - d0, 4.0 * d0 - dm1, dm1, d0);
  } else {
    dhp = minmod2(d0, dp1);
    dhm = minmod2(dm1, d0);
  }
  T fi = F(0), fip = F(1), fim = F(-1);
  T f_ul = fi + S.mp_alpha * (fi - fim);
  T f_md = 0.5 * (fi + fip) - 0.5 * dhp;
  T f_lc = fi + 0.5 * (fi - fim) + S.mp_beta / 3.0 * dhm;
  *fmin = max_(min3(fi, fip, f_md), min3(fi, f_ul, f_lc));
  *fmax = min_(max3(fi, fip, f_md), max3(fi, f_ul, f_lc));
}

/* TVD5 flux of Eqs. high order TVD, TVDhighorder2, TVDbeta (alpha = 2).
   Reading: written without divisions.  With D_m = f_m - f_{m-1}:
   r_j = D_{i+1}/D_i, 1/r_{j-1} = D_{i-1}/D_i, r_j r_{j+1} = D_{i+2}/D_i, so
   phi*delta^- = max(0, min(2 D_i, 2 D_{i+1}, B)) when D_i > 0,
               = min(0, max(2 D_i, 2 D_{i+1}, B)) when D_i < 0,
               = 0 when D_i = 0 (the limit; phi is bounded by alpha),
   B = (-2 D_{i-1} + 11 D_i + 24 D_{i+1} - 3 D_{i+2}) / 30.
   Equal to the printed formula wherever that is defined (checked by the tests). */
template <class T, class FN>
inline T tvd5_flux(FN F) {
  T Dm = F(-1) - F(-2), D0 = F(0) - F(-1), Dp = F(1) - F(0), Dpp = F(2) - F(1);
  T B = (-2.0 * Dm + 11.0 * D0 + 24.0 * Dp - 3.0 * Dpp) / 30.0;
  T phid;
  double s = sgn(D0);
  if (s > 0) phid = max_(T(0.0), min3(2.0 * D0, 2.0 * Dp, B));
  else if (s < 0) phid = min_(T(0.0), max3(2.0 * D0, 2.0 * Dp, B));
  else phid = 0.0;
  return F(0) + 0.5 * phid;
}

/* Van Albada flux, Eqs. van_Albada_limiter, slop_ratio, vAflux, kappa = 1/3.
   Reading: phi = 2 r/(r^2+1) with r = delta^+/delta^- written as
   2 delta^+ delta^- / (delta^+^2 + delta^-^2) (0 when both vanish). */
template <class T, class FN>
inline T va_flux(FN F) {
  T dm = F(0) - F(-1), dp = F(1) - F(0);
  T den = dp * dp + dm * dm;
  T phi = 0.0;
  if (val(den) > 0) phi = 2.0 * dp * dm / den;
  const double kappa = 1.0 / 3.0;
  return F(0) + phi / 4.0 * ((1.0 - kappa * phi) * dm + (1.0 + kappa * phi) * dp);
}

/* ------------------------------------------------------------------ TENO-M */
/* Adaptive cutoff of TENO8A (Section 2.4): returns [beta] and C_T = 10^{-[beta]}.
   Reading: eta is evaluated on the sequence being reconstructed. */
template <class T, class FN>
inline double adaptive_ct(FN F, int* ct_exp, double* beta_out) {
  const double xi = 1e-3, Cr = 0.23, a1 = 10.5, a2 = 3.5;
  const double eps = 0.9 * Cr / (1.0 - 0.9 * Cr) * xi * xi;
  T eta[4];
  for (int q = 0; q < 4; ++q) {
    int c = q - 1;  /* eta_{i-1}, eta_i, eta_{i+1}, eta_{i+2} */
    T dfp = F(c + 1) - F(c), dfm = F(c) - F(c - 1);
    eta[q] = (abs_(2.0 * dfp * dfm) + eps) / (dfp * dfp + dfm * dfm + eps);
  }
  T eh = min_(min_(eta[0], eta[1]), min_(eta[2], eta[3]));
  T m = 1.0 - min_(T(1.0), eh / Cr);
  T om = 1.0 - m;
  T g = om * om * om * om * (1.0 + 4.0 * m);
  T beta = a1 - a2 * (1.0 - g);
  double bv = val(beta);
  int e = (int)std::floor(bv);
  *ct_exp = e;
  *beta_out = bv;
  /* reading: [beta] lies in {7,8,9,10}; C_T from the literal decimal table */
  static const double tab[4] = {1e-7, 1e-8, 1e-9, 1e-10};
  int idx = e - 7;
  if (idx < 0) idx = 0;
  if (idx > 3) idx = 3;
  return tab[idx];
}

/* One scalar TENO-M reconstruction of h at x_{i+1/2} (Sections 2-3).
   F(m) returns f_{i+m} for m = -K/2+1 .. K/2. */
template <class T, class FN>
inline T teno_m(const Scheme& S, FN F, ReconDiag* diag) {
  const int K = S.K, nk = K - 2;
  const double C = 1.0, eps = 1e-40;  /* Eq. measureTENO: C = 1, q = 6, epsilon = 1e-40 */
  T fk[6], bk[6], gk[6];
  for (int k = 0; k < nk; ++k) fk[k] = candidate<T>(k, F);      /* Table 1 */
  for (int k = 0; k < nk; ++k) bk[k] = beta_candidate<T>(k, F); /* beta_{k,r} */
  T bK = beta_full<T>(K, F);
  T tau = abs_(bK - (bk[1] + bk[2] + 4.0 * bk[0]) / 6.0);     /* Eq. taukTENO */
  T sum = 0.0;
  for (int k = 0; k < nk; ++k) {
    T x = C + tau / (bk[k] + eps);
    gk[k] = x * x * x * x * x * x;                              /* (.)^q, q = 6 */
    sum = sum + gk[k];
  }
  double CT;
  int ct_exp = 0;
  double beta_ct = 0.0;
  if (S.ct_mode == CT_ADAPTIVE) CT = adaptive_ct<T>(F, &ct_exp, &beta_ct);
  else CT = S.ct_const;
  int bits = 0, nonfinite = 0;
  for (int k = 0; k < nk; ++k) {
    T chi = gk[k] / sum;                                         /* Eq. normalize */
    if (!std::isfinite(val(chi)) || !std::isfinite(val(gk[k]))) nonfinite = 1;
    int delta = lt(chi, T(CT)) ? 0 : 1;                          /* Eq. cut-off (tie -> 1) */
    bits |= delta << k;
    if (diag) diag->cut_rel[k] = (val(chi) - CT) / CT;
  }
  if (diag) {
    diag->delta_bits = bits;
    diag->ct_exp = ct_exp;
    diag->beta_ct = beta_ct;
    diag->nonfinite = nonfinite;
  }
  if (S.weights == W_TENO) {                                     /* Eqs. weight_renormalize, reconstuction */
    T num = 0.0, den = 0.0;
    for (int k = 0; k < nk; ++k)
      if (bits >> k & 1) { num = num + S.d[k] * fk[k]; den = den + S.d[k]; }
    return num / den;
  }
  /* Eq. mp_flux: filter the nonsmooth candidates */
  if (bits != (1 << nk) - 1) {
    if (S.limiter == LIM_MP) {
      T fmin, fmax;
      mp_bounds<T>(S, F, &fmin, &fmax);
      for (int k = 0; k < nk; ++k)
        if (!(bits >> k & 1)) fk[k] = median(fk[k], fmin, fmax);  /* Eq. value_monotonicity_preserving */
    } else {
      T flim = (S.limiter == LIM_TVD5) ? tvd5_flux<T>(F) : va_flux<T>(F);
      for (int k = 0; k < nk; ++k)
        if (!(bits >> k & 1)) fk[k] = flim;  /* one fixed limited flux (Section 3.2.3) */
    }
  }
  T f = 0.0;
  for (int k = 0; k < nk; ++k) f = f + S.d[k] * fk[k];          /* Eq. reconstuction, w_k = d_k */
  return f;
}

/* ------------------------------------------------------------------ Euler */
struct Grid {
  int dim;
  int n[3];
  double dx[3];
  int bc[3];
  double gamma;
};

inline long long ncell(const Grid& g) {
  long long c = 1;
  for (int a = 0; a < g.dim; ++a) c *= g.n[a];
  return c;
}

/* Cell index with boundary condition applied along axis a (periodic wrap or
   zero-gradient copy; reading: the paper does not state how ghosts are filled). */
inline int bc_index(const Grid& g, int a, int j) {
  int n = g.n[a];
  if (g.bc[a] == BC_PERIODIC) return ((j % n) + n) % n;
  return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

/* Point quantities of the Euler equations (Section 4: compressible Euler). */
template <class T> struct Point {
  T U[5];
  T rho, vel[3], p, c, H;
};

template <class T>
inline void point_from_U(const Grid& g, const T* U, Point<T>* P) {
  const int D = g.dim, nv = D + 2;
  for (int q = 0; q < nv; ++q) P->U[q] = U[q];
  P->rho = U[0];
  T ke = 0.0;
  for (int d = 0; d < D; ++d) {
    P->vel[d] = U[1 + d] / U[0];
    ke = ke + U[1 + d] * P->vel[d];
  }
  P->p = (g.gamma - 1.0) * (U[nv - 1] - 0.5 * ke);
  P->c = sqrt_(g.gamma * P->p / P->rho);
  P->H = (U[nv - 1] + P->p) / P->rho;
}

/* physical flux F_a(U) */
template <class T>
inline void phys_flux(const Grid& g, const Point<T>& P, int a, T* F) {
  const int D = g.dim, nv = D + 2;
  T un = P.vel[a];
  F[0] = P.U[0] * un;
  for (int d = 0; d < D; ++d) F[1 + d] = P.U[1 + d] * un + (d == a ? P.p : T(0.0));
  F[nv - 1] = (P.U[nv - 1] + P.p) * un;
}

/* Roe-averaged eigensystem at a face for axis a.  Reading: the fixed textbook basis
   (u-c, entropy, unit tangential shear waves in increasing axis order, u+c); the
   paper names Roe averaging and characteristic decomposition only (Section 4). */
template <class T>
struct Eigen {
  T R[5][5];  /* columns r_s */
  T L[5][5];  /* rows l_s */
  T lam_dummy;
  int bad;    /* c^2 <= 0 */
};

template <class T>
inline void roe_eigen(const Grid& g, const Point<T>& PL, const Point<T>& PR, int a, Eigen<T>* E) {
  const int D = g.dim, nv = D + 2;
  T sL = sqrt_(PL.rho), sR = sqrt_(PR.rho);
  T u[3];
  T q2 = 0.0;
  for (int d = 0; d < D; ++d) {
    u[d] = (sL * PL.vel[d] + sR * PR.vel[d]) / (sL + sR);
    q2 = q2 + u[d] * u[d];
  }
  T H = (sL * PL.H + sR * PR.H) / (sL + sR);
  T c2 = (g.gamma - 1.0) * (H - 0.5 * q2);
  E->bad = val(c2) <= 0;
  T c = sqrt_(c2);
  int tang[2], nt = 0;
  for (int d = 0; d < D; ++d)
    if (d != a) tang[nt++] = d;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) { E->R[i][j] = 0.0; E->L[i][j] = 0.0; }
  /* right eigenvectors (columns) */
  const int sm = 0, se = 1, sp = nv - 1;
  E->R[0][sm] = 1.0; E->R[0][se] = 1.0; E->R[0][sp] = 1.0;
  for (int d = 0; d < D; ++d) {
    T en = (d == a) ? T(1.0) : T(0.0);
    E->R[1 + d][sm] = u[d] - c * en;
    E->R[1 + d][se] = u[d];
    E->R[1 + d][sp] = u[d] + c * en;
  }
  E->R[nv - 1][sm] = H - u[a] * c;
  E->R[nv - 1][se] = 0.5 * q2;
  E->R[nv - 1][sp] = H + u[a] * c;
  for (int t = 0; t < nt; ++t) {
    int s = 2 + t, dt = tang[t];
    E->R[0][s] = 0.0;
    for (int d = 0; d < D; ++d) E->R[1 + d][s] = (d == dt) ? T(1.0) : T(0.0);
    E->R[nv - 1][s] = u[dt];
  }
  /* left eigenvectors (rows), L = R^{-1} in closed form */
  T b1 = (g.gamma - 1.0) / c2;
  T b2 = 0.5 * q2 * b1;
  T ua_c = u[a] / c;
  E->L[sm][0] = 0.5 * (b2 + ua_c);
  E->L[se][0] = 1.0 - b2;
  E->L[sp][0] = 0.5 * (b2 - ua_c);
  for (int d = 0; d < D; ++d) {
    T en_c = (d == a) ? T(1.0) / c : T(0.0);
    E->L[sm][1 + d] = 0.5 * (-b1 * u[d] - en_c);
    E->L[se][1 + d] = b1 * u[d];
    E->L[sp][1 + d] = 0.5 * (-b1 * u[d] + en_c);
  }
  E->L[sm][nv - 1] = 0.5 * b1;
  E->L[se][nv - 1] = -b1;
  E->L[sp][nv - 1] = 0.5 * b1;
  for (int t = 0; t < nt; ++t) {
    int s = 2 + t, dt = tang[t];
    E->L[s][0] = -u[dt];
    for (int d = 0; d < D; ++d) E->L[s][1 + d] = (d == dt) ? T(1.0) : T(0.0);
    E->L[s][nv - 1] = 0.0;
  }
}

/* Per-face diagnostics of a system face. */
struct FaceDiag {
  uint8_t flags[5][2];    /* per field, per side (0 = f+, 1 = f-): delta bits | ct code << 6 */
  double cut[5][2];       /* min over k of |chi_k - C_T| / C_T, and (adaptive C_T) of the
                             relative distance of beta to the nearest integer */
  double noise[5][2];     /* rounding-noise ratio of the sequence: 2^-52 max|g_m| over
                             max|g_m - g_i| (0 for an exactly constant sequence); where it
                             is large the cutoff decision is set by rounding, not data */
  double scale[5];        /* per component, sum over fields s of |R_{v,s}| (|f+_s| + |f-_s|):
                             the magnitude of the terms of the back-projection sum */
  int nonphysical;
};

/* Rounding-noise ratio of a K-point sequence (diagnostic only): the largest, over the
   candidate stencils and the full stencil, of 2^-52 max|g| / (spread of the stencil's
   values about g_i); infinite when a stencil's values are all equal.  Where it is large,
   some beta_k is made of rounding noise and the cutoff decision is set by rounding. */
template <class T>
inline double noise_ratio(const T* g, int K) {
  const int h = K / 2;
  double mx = 0.0;
  for (int q = 0; q < K; ++q) mx = std::fmax(mx, std::fabs(val(g[q])));
  const int j0s[7] = {ORC_S0_J0, ORC_S1_J0, ORC_S2_J0, ORC_S3_J0, ORC_S4_J0, ORC_S5_J0,
                      K == 6 ? ORC_F6_J0 : ORC_F8_J0};
  const int rs[7] = {ORC_S0_R, ORC_S1_R, ORC_S2_R, ORC_S3_R, ORC_S4_R, ORC_S5_R, K == 6 ? ORC_F6_R : ORC_F8_R};
  const double gi = val(g[h - 1]);
  double worst = 0.0;
  for (int k = 0; k < 7; ++k) {
    if (k < 6 && k >= K - 2) continue;
    double dv = 0.0;
    for (int m = 0; m < rs[k]; ++m) dv = std::fmax(dv, std::fabs(val(g[j0s[k] + m + h - 1]) - gi));
    double r = (dv == 0.0) ? (mx == 0.0 ? 0.0 : HUGE_VAL) : 2.220446049250313e-16 * mx / dv;
    worst = std::fmax(worst, r);
  }
  return worst;
}

/* Numerical flux at face f (between cells f-1 and f) along axis a of the pencil whose
   other indices are fixed in `base` (cell multi-index; base[a] is ignored).
   Characteristic decomposition with Roe averages + Rusanov (local Lax-Friedrichs)
   splitting (Section 4), scalar TENO-M per field and side (Sections 2-3).
   Reading: alpha_s = max over the K stencil points of |lambda_s(U_m)|; the f^- side is
   reconstructed on the stencil mirrored about x_{i+1/2}. */
template <class T>
inline void face_flux(const Grid& g, const Scheme& S, const T* U, int a, const int* base, int f,
                      T* Fhat, FaceDiag* diag) {
  const int D = g.dim, nv = D + 2, K = S.K, h = K / 2;
  long long nc = ncell(g);
  long long stride[3] = {1, g.n[0], (long long)g.n[0] * (g.n[1] > 0 ? g.n[1] : 1)};
  int i = f - 1;
  /* stencil points m = i-h+1 .. i+h (K points) */
  Point<T> P[8];
  T Fm[8][5];
  for (int q = 0; q < K; ++q) {
    int j = bc_index(g, a, i - h + 1 + q);
    long long lin = 0;
    for (int d = 0; d < D; ++d) lin += (long long)((d == a) ? j : base[d]) * stride[d];
    T Uc[5];
    for (int v = 0; v < nv; ++v) Uc[v] = U[v * nc + lin];
    point_from_U(g, Uc, &P[q]);
    phys_flux(g, P[q], a, Fm[q]);
  }
  Eigen<T> E;
  roe_eigen(g, P[h - 1], P[h], a, &E);
  if (diag) diag->nonphysical = E.bad;
  for (int q = 0; q < K; ++q)
    if (diag && (val(P[q].p) <= 0 || val(P[q].rho) <= 0)) diag->nonphysical = 1;
  T fsum[5];
  double fabs_sum[5] = {0, 0, 0, 0, 0};
  for (int s = 0; s < nv; ++s) {
    /* characteristic variables and fluxes of field s at the K points */
    T W[8], G[8], lam[8];
    for (int q = 0; q < K; ++q) {
      T w = 0.0, gg = 0.0;
      for (int v = 0; v < nv; ++v) {
        w = w + E.L[s][v] * P[q].U[v];
        gg = gg + E.L[s][v] * Fm[q][v];
      }
      W[q] = w;
      G[q] = gg;
      T un = P[q].vel[a];
      lam[q] = (s == 0) ? un - P[q].c : (s == nv - 1 ? un + P[q].c : un);
    }
    T alpha = abs_(lam[0]);
    for (int q = 1; q < K; ++q) alpha = max_(alpha, abs_(lam[q]));
    T gp[8], gm[8];
    for (int q = 0; q < K; ++q) {
      gp[q] = 0.5 * (G[q] + alpha * W[q]);
      gm[q] = 0.5 * (G[q] - alpha * W[q]);
    }
    ReconDiag dp, dm;
    /* f+ : F(m) = g+_{i+m} ; index of point i+m in the stencil is m + h - 1 */
    T fplus = teno_m<T>(S, [&](int m) { return gp[m + h - 1]; }, &dp);
    /* f- : mirrored about x_{i+1/2}: F(m) = g-_{i+1-m} */
    T fminus = teno_m<T>(S, [&](int m) { return gm[h - m]; }, &dm);
    fsum[s] = fplus + fminus;
    if (diag) {
      fabs_sum[s] = std::fabs(val(fplus)) + std::fabs(val(fminus));
      ReconDiag* dd[2] = {&dp, &dm};
      T gmr[8];  /* the f- sequence in the mirrored order it is reconstructed in */
      for (int q = 0; q < K; ++q) gmr[q] = gm[K - 1 - q];
      const T* seq[2] = {gp, gmr};
      for (int side = 0; side < 2; ++side) {
        int code = (S.ct_mode == CT_ADAPTIVE) ? (dd[side]->ct_exp - 7) & 3 : 0;
        diag->flags[s][side] = (uint8_t)(dd[side]->delta_bits | (code << 6));
        double c = 1e300;
        for (int k = 0; k < K - 2; ++k) c = std::fmin(c, std::fabs(dd[side]->cut_rel[k]));
        if (S.ct_mode == CT_ADAPTIVE) {
          double b = dd[side]->beta_ct;
          c = std::fmin(c, std::fabs(b - std::floor(b + 0.5)) / b);
        }
        diag->cut[s][side] = c;
        diag->noise[s][side] = noise_ratio(seq[side], K);
        if (dd[side]->nonfinite) diag->nonphysical = 1;
      }
    }
  }
  /* back-projection F = sum_s r_s (f+_s + f-_s) */
  for (int v = 0; v < nv; ++v) {
    T acc = 0.0;
    double sc = 0.0;
    for (int s = 0; s < nv; ++s) {
      acc = acc + E.R[v][s] * fsum[s];
      sc += std::fabs(val(E.R[v][s])) * fabs_sum[s];
    }
    Fhat[v] = acc;
    if (diag) diag->scale[v] = sc;
  }
}

/* Face layout for axis a: [nv][faces], faces indexed like cells but with n[a]+1 entries
   along axis a (face f lies between cells f-1 and f). */
inline long long nface(const Grid& g, int a) {
  long long c = 1;
  for (int d = 0; d < g.dim; ++d) c *= (d == a) ? g.n[d] + 1 : g.n[d];
  return c;
}

/* All faces of axis a.  Fhat: [nv][nface]; flags, cut, noise: [nface][nv][2] (each may
   be null; see FaceDiag). */
template <class T>
inline int all_faces(const Grid& g, const Scheme& S, const T* U, int a, T* Fhat, uint8_t* flags,
                     double* cut, double* noise, double* scale = nullptr) {
  const int D = g.dim, nv = D + 2;
  int fn[3] = {1, 1, 1};
  for (int d = 0; d < D; ++d) fn[d] = (d == a) ? g.n[d] + 1 : g.n[d];
  long long nf = nface(g, a);
  int bad = 0;
  for (int z = 0; z < fn[2]; ++z)
    for (int y = 0; y < fn[1]; ++y)
      for (int x = 0; x < fn[0]; ++x) {
        int idx[3] = {x, y, z};
        long long lin = x + (long long)fn[0] * (y + (long long)fn[1] * z);
        T F[5];
        FaceDiag dg;
        face_flux<T>(g, S, U, a, idx, idx[a], F, &dg);
        for (int v = 0; v < nv; ++v) {
          Fhat[v * nf + lin] = F[v];
          if (scale) scale[v * nf + lin] = dg.scale[v];
        }
        for (int v = 0; v < nv; ++v)
          for (int s = 0; s < 2; ++s) {
            long long o = (lin * nv + v) * 2 + s;
            if (flags) flags[o] = dg.flags[v][s];
            if (cut) cut[o] = dg.cut[v][s];
            if (noise) noise[o] = dg.noise[v][s];
          }
        bad |= dg.nonphysical;
      }
  return bad;
}

/* ------------------------------------------------------------------ positivity */
/* Pressure (gamma - 1) (E - |m|^2 / (2 rho)) of one conserved state. */
inline double pressure_of(const Grid& g, const double* W) {
  const int nv = g.dim + 2;
  double m2 = 0.0;
  for (int d = 0; d < g.dim; ++d) m2 += W[1 + d] * W[1 + d];
  return (g.gamma - 1.0) * (W[nv - 1] - 0.5 * m2 / W[0]);
}

/* Positivity-preserving flux limiter that Section 4.4 applies (Hu, Adams & Shu,
   J. Comput. Phys. 242, 2013), for one forward-Euler stage of length dt, on the face
   fluxes Fh ([nv][nface]) of axis a computed from U.
   The stage update U_i - sum_a lambda_a (F_{a,i+1/2} - F_{a,i-1/2}), lambda_a = dt/dx_a,
   is the mean of the 2D one-sided states U_i - mu_a F_{a,i+1/2} and U_i + mu_a F_{a,i-1/2}
   with mu_a = 2 D lambda_a; each stays admissible when its face flux is the first-order
   Lax-Friedrichs flux F^LF = (F(U_L) + F(U_R) - alpha (U_R - U_L)) / 2 and the step is small
   enough.  The face flux becomes F^LF + theta (F^H - F^LF), F^H the high-order flux:
     theta_rho: on each side, if the density of the one-sided state made with F^H is below
       eps = min(1e-13, density made with F^LF), the theta at which the (linear) density
       equals eps; the smaller of the two sides, else 1;
     theta_p: the same for the pressure, with F^H replaced by the density-limited flux
       F1 = F^LF + theta_rho (F^H - F^LF); the pressure is concave in the state, so the
       theta where (1 - theta) p(F^LF state) + theta p(F1 state) = eps keeps it >= eps;
     flux = F^LF + theta_p (F1 - F^LF);
   theta = 1 leaves the flux it would scale as it is (no rounding of an unlimited face).
   Readings: alpha = max of |u_a| + c over the two cells of the face (local Lax-Friedrichs);
   eps as above; the 1/(2D) split; the outside cell of a transmissive boundary face (the
   boundary's copy of the edge cell) is checked like an interior one. */
inline void positivity_limit(const Grid& g, const double* U, int a, double dt, double* Fh) {
  const int D = g.dim, nv = D + 2;
  const long long nc = ncell(g), nf = nface(g, a);
  const long long stride[3] = {1, g.n[0], (long long)g.n[0] * g.n[1]};
  int fn[3] = {1, 1, 1};
  for (int d = 0; d < D; ++d) fn[d] = (d == a) ? g.n[d] + 1 : g.n[d];
  const double mu = 2.0 * D * dt / g.dx[a];
  for (int z = 0; z < fn[2]; ++z)
    for (int y = 0; y < fn[1]; ++y)
      for (int x = 0; x < fn[0]; ++x) {
        const int idx[3] = {x, y, z};
        const long long lin = x + (long long)fn[0] * (y + (long long)fn[1] * z);
        double Us[2][5], Fc[2][5], sp[2];
        for (int side = 0; side < 2; ++side) {
          const int j = bc_index(g, a, idx[a] - 1 + side); /* cell left (0) or right (1) of the face */
          long long cl = 0;
          for (int d = 0; d < D; ++d) cl += (long long)((d == a) ? j : idx[d]) * stride[d];
          for (int v = 0; v < nv; ++v) Us[side][v] = U[v * nc + cl];
          Point<double> P;
          point_from_U(g, Us[side], &P);
          phys_flux(g, P, a, Fc[side]);
          sp[side] = std::fabs(P.vel[a]) + P.c;
        }
        const double alpha = std::fmax(sp[0], sp[1]);
        double FLF[5], FH[5], F1[5];
        for (int v = 0; v < nv; ++v) {
          FLF[v] = 0.5 * (Fc[0][v] + Fc[1][v] - alpha * (Us[1][v] - Us[0][v]));
          FH[v] = Fh[v * nf + lin];
        }
        const double sgn_mu[2] = {-mu, mu}; /* left cell loses F, right cell gains it */
        double th = 1.0;
        for (int side = 0; side < 2; ++side) {
          const double rlf = Us[side][0] + sgn_mu[side] * FLF[0];
          const double rh = Us[side][0] + sgn_mu[side] * FH[0];
          const double eps = std::fmin(1e-13, rlf);
          if (rh < eps) th = std::fmin(th, (rlf - eps) / (rlf - rh));
        }
        for (int v = 0; v < nv; ++v) F1[v] = (th == 1.0) ? FH[v] : FLF[v] + th * (FH[v] - FLF[v]);
        double tp = 1.0;
        for (int side = 0; side < 2; ++side) {
          double Wlf[5], W1[5];
          for (int v = 0; v < nv; ++v) {
            Wlf[v] = Us[side][v] + sgn_mu[side] * FLF[v];
            W1[v] = Us[side][v] + sgn_mu[side] * F1[v];
          }
          const double plf = pressure_of(g, Wlf), p1 = pressure_of(g, W1);
          const double eps = std::fmin(1e-13, plf);
          if (p1 < eps) tp = std::fmin(tp, (plf - eps) / (plf - p1));
        }
        if (tp < 1.0 || th < 1.0)
          for (int v = 0; v < nv; ++v) Fh[v * nf + lin] = (tp == 1.0) ? F1[v] : FLF[v] + tp * (F1[v] - FLF[v]);
      }
}

/* Semi-discrete operator dU/dt = -sum_a (F_{a,i+1/2} - F_{a,i-1/2}) / dx_a
   (Eq. approximateEq, dimension by dimension as in Section 4).  With pp_dt > 0 and
   S.positivity set, the face fluxes first pass the positivity limiter of a forward-Euler
   stage of length pp_dt (FP64 only). */
template <class T>
inline int rhs(const Grid& g, const Scheme& S, const T* U, T* dUdt, double pp_dt = 0.0) {
  const int D = g.dim, nv = D + 2;
  long long nc = ncell(g);
  for (long long q = 0; q < nv * nc; ++q) dUdt[q] = 0.0;
  int bad = 0;
  for (int a = 0; a < D; ++a) {
    long long nf = nface(g, a);
    std::vector<T> Fh((size_t)nv * nf);
    bad |= all_faces<T>(g, S, U, a, Fh.data(), nullptr, nullptr, nullptr);
    if constexpr (std::is_same<T, double>::value)
      if (S.positivity && pp_dt > 0.0) positivity_limit(g, U, a, pp_dt, Fh.data());
    int fn[3] = {1, 1, 1};
    for (int d = 0; d < D; ++d) fn[d] = (d == a) ? g.n[d] + 1 : g.n[d];
    long long fstride = 1;
    for (int d = 0; d < a; ++d) fstride *= fn[d];
    int cn[3] = {1, 1, 1};
    for (int d = 0; d < D; ++d) cn[d] = g.n[d];
    for (int z = 0; z < cn[2]; ++z)
      for (int y = 0; y < cn[1]; ++y)
        for (int x = 0; x < cn[0]; ++x) {
          long long c = x + (long long)cn[0] * (y + (long long)cn[1] * z);
          long long fl = x + (long long)fn[0] * (y + (long long)fn[1] * z); /* face i-1/2 */
          long long fr = fl + fstride;                                      /* face i+1/2 */
          for (int v = 0; v < nv; ++v)
            dUdt[v * nc + c] = dUdt[v * nc + c] - (Fh[v * nf + fr] - Fh[v * nf + fl]) / g.dx[a];
        }
  }
  return bad;
}

/* Conserved state from primitives (rho, u_1..u_D, p). */
template <class T>
inline void init_state(const Grid& g, const T* prim, T* U) {
  const int D = g.dim, nv = D + 2;
  long long nc = ncell(g);
  for (long long c = 0; c < nc; ++c) {
    T rho = prim[c];
    T ke = 0.0;
    for (int d = 0; d < D; ++d) {
      T u = prim[(1 + d) * nc + c];
      U[(1 + d) * nc + c] = rho * u;
      ke = ke + rho * u * u;
    }
    U[c] = rho;
    U[(nv - 1) * nc + c] = prim[(nv - 1) * nc + c] / (g.gamma - 1.0) + 0.5 * ke;
  }
}

/* Largest stable step: dt = CFL / max_i sum_a (|u_a| + c)_i / dx_a  (Section 4, CFL 0.4).
   Reading: the multi-dimensional signal-speed sum. */
inline double max_dt(const Grid& g, const double* U, double cfl) {
  const int D = g.dim;
  long long nc = ncell(g);
  double smax = 0.0;
  for (long long c = 0; c < nc; ++c) {
    double Uc[5];
    for (int v = 0; v < D + 2; ++v) Uc[v] = U[v * nc + c];
    Point<double> P;
    point_from_U(g, Uc, &P);
    double s = 0.0;
    for (int a = 0; a < D; ++a) s += (std::fabs(P.vel[a]) + P.c) / g.dx[a];
    if (s > smax) smax = s;
  }
  return cfl / smax;
}

/* Third-order SSP Runge-Kutta step (Gottlieb-Shu-Tadmor, named in Section 4):
   U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1)); U^{n+1} = 1/3 U + 2/3 (U2 + dt L(U2)). */
template <class T>
inline int rk3_step(const Grid& g, const Scheme& S, T* U, T dt) {
  const int nv = g.dim + 2;
  long long N = nv * ncell(g);
  std::vector<T> L(N), U1(N), U2(N);
  /* each stage is a forward-Euler step of length dt (the positivity limiter's lambda) */
  int bad = rhs<T>(g, S, U, L.data(), val(dt));
  for (long long q = 0; q < N; ++q) U1[q] = U[q] + dt * L[q];
  bad |= rhs<T>(g, S, U1.data(), L.data(), val(dt));
  for (long long q = 0; q < N; ++q) U2[q] = 0.75 * U[q] + 0.25 * (U1[q] + dt * L[q]);
  bad |= rhs<T>(g, S, U2.data(), L.data(), val(dt));
  for (long long q = 0; q < N; ++q) U[q] = 1.0 / 3.0 * U[q] + 2.0 / 3.0 * (U2[q] + dt * L[q]);
  return bad;
}

/* ------------------------------------------------------------------ scalar advection */
/* Linear advection u_t + u_x = 0 (Section 4.1), periodic: f = u, alpha = 1, so
   f+ = u and f- = 0; the conservative difference of Eq. approximateEq. */
template <class T>
inline void scalar_rhs(const Scheme& S, int n, double dx, const T* u, T* dudt) {
  const int h = S.K / 2;
  std::vector<T> fh(n + 1);
  for (int f = 0; f <= n; ++f) {
    int i = f - 1;
    T gp[8], gm[8];
    for (int q = 0; q < S.K; ++q) {
      int j = (((i - h + 1 + q) % n) + n) % n;
      T fu = u[j];
      gp[q] = 0.5 * (fu + 1.0 * u[j]);
      gm[q] = 0.5 * (fu - 1.0 * u[j]);
    }
    T a = teno_m<T>(S, [&](int m) { return gp[m + h - 1]; }, nullptr);
    T b = teno_m<T>(S, [&](int m) { return gm[h - m]; }, nullptr);
    fh[f] = a + b;
  }
  for (int c = 0; c < n; ++c) dudt[c] = -(fh[c + 1] - fh[c]) / dx;
}

template <class T>
inline void scalar_rk3(const Scheme& S, int n, double dx, T* u, double dt) {
  std::vector<T> L(n), u1(n), u2(n);
  scalar_rhs<T>(S, n, dx, u, L.data());
  for (int q = 0; q < n; ++q) u1[q] = u[q] + dt * L[q];
  scalar_rhs<T>(S, n, dx, u1.data(), L.data());
  for (int q = 0; q < n; ++q) u2[q] = 0.75 * u[q] + 0.25 * (u1[q] + dt * L[q]);
  scalar_rhs<T>(S, n, dx, u2.data(), L.data());
  for (int q = 0; q < n; ++q) u[q] = 1.0 / 3.0 * u[q] + 2.0 / 3.0 * (u2[q] + dt * L[q]);
}

}  // namespace orc
