/* Frozen-branch linearisation of the face flux (adjoint of Sections 2-4 with every branch
 * taken from the forward pass).
 *
 * TENO-M assembles the candidates with constant weights w_k = d_k (Section 3.3), so once the
 * cutoff flags delta_k and the limiter's selections are fixed, the reconstruction is a LINEAR
 * function of the K stencil values: fhat = sum_q omega_q v_q.  teno_m_weights() replays the
 * forward's decisions on the same values (same expressions, same integer-pipe comparisons)
 * and returns omega.  No derivative flows through beta, tau, gamma or chi.
 *
 * face_vjp_smem() is the reverse-mode derivative of face_flux_smem(): given the adjoint Fbar
 * of one face flux it returns, for each of the K stencil points, the adjoint of the point's
 * conserved state, through the back-projection, the frozen reconstructions, the LLF split
 * (alpha's argmax frozen), the characteristic projection, the Roe-averaged eigenvectors and
 * the point quantities (primitives, physical flux). */
#pragma once
#include "tenom_face.cuh"

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

/* Table 1 coefficients on v (index c = f_i) */
template <int K>
__device__ __forceinline__ void cand_coeffs(int k, double* g) {
  constexpr int c = K / 2 - 1;
#pragma unroll
  for (int i = 0; i < K; ++i) g[i] = 0.0;
  switch (k) {
    case 0: g[c - 1] = -1.0 / 6.0; g[c] = 5.0 / 6.0; g[c + 1] = 2.0 / 6.0; break;
    case 1: g[c] = 2.0 / 6.0; g[c + 1] = 5.0 / 6.0; g[c + 2] = -1.0 / 6.0; break;
    case 2: g[c - 2] = 2.0 / 6.0; g[c - 1] = -7.0 / 6.0; g[c] = 11.0 / 6.0; break;
    case 3: g[c] = 3.0 / 12.0; g[c + 1] = 13.0 / 12.0; g[c + 2] = -5.0 / 12.0; g[c + 3] = 1.0 / 12.0; break;
    case 4: g[c - 3] = -3.0 / 12.0; g[c - 2] = 13.0 / 12.0; g[c - 1] = -23.0 / 12.0; g[c] = 25.0 / 12.0; break;
    default:
      g[c] = 12.0 / 60.0; g[c + 1] = 77.0 / 60.0; g[c + 2] = -43.0 / 60.0; g[c + 3] = 17.0 / 60.0;
      g[c + 4] = -3.0 / 60.0;
      break;
  }
}

/* omega with fhat = sum_q omega_q v_q under the frozen flags (delta bits in `bits`) */
template <int K>
__device__ __forceinline__ void central_weights(double (&om)[K]) {
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

/* Reverse of the point quantities (stage_point): adjoints of the physical flux F_AXIS (Fb),
   of the velocity (velb), sound speed (cb), enthalpy (Hb) and sqrt(rho) (sb) of one point
   -> adjoint of its conserved state, added to Ub. */
template <int NV, int AXIS>
__device__ __forceinline__ void point_vjp(const double* sm, const double* rec, int NP, int p, double gamma,
                                          const double (&Fb)[NV], double (&velb)[NV - 2], double cb, double Hb,
                                          double sb, double* Ub, int ustride) {
  using L = PointLayout<NV>;
  constexpr int D = NV - 2;
  const double rho = sm[L::cU * NP + p], E = sm[(L::cU + NV - 1) * NP + p];
  double m[D], vel[D], ke = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    m[d] = sm[(L::cU + 1 + d) * NP + p];
    vel[d] = sm[(L::cV + d) * NP + p];
    ke += m[d] * vel[d];
  }
  const double pr = (gamma - 1.0) * (E - 0.5 * ke);
  const double H = sm[L::cH * NP + p], c = sm[L::cC * NP + p];
  const double un = vel[AXIS];
  const double rinv = rec[p];                 /* 1/rho */
  double rhob = 0.0, Eb = 0.0, pb = 0.0, mb[D];
#pragma unroll
  for (int d = 0; d < D; ++d) mb[d] = 0.0;
  /* physical flux F = (rho un, m un + p e_a, (E + p) un) */
  double unb = rho * Fb[0];
  rhob += un * Fb[0];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    mb[d] += un * Fb[1 + d];
    unb += m[d] * Fb[1 + d];
  }
  pb += Fb[1 + AXIS];
  Eb += un * Fb[NV - 1];
  pb += un * Fb[NV - 1];
  unb += (E + pr) * Fb[NV - 1];
  velb[AXIS] += unb;
  /* H = (E + p)/rho */
  Eb += Hb * rinv;
  pb += Hb * rinv;
  rhob -= H * Hb * rinv;
  /* c = sqrt(gamma p / rho) */
  const double k = cb * rec[NP + p];          /* 1/(2 c rho) */
  pb += gamma * k;
  rhob -= c * c * k;
  /* sqrt(rho) */
  rhob += sb * rec[2 * NP + p];               /* 1/(2 sqrt(rho)) */
  /* p = (gamma - 1)(E - ke/2), ke = sum m_d vel_d */
  Eb += (gamma - 1.0) * pb;
  const double keb = -0.5 * (gamma - 1.0) * pb;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    mb[d] += vel[d] * keb;
    velb[d] += m[d] * keb;
  }
  /* vel_d = m_d / rho */
#pragma unroll
  for (int d = 0; d < D; ++d) {
    mb[d] += velb[d] * rinv;
    rhob -= vel[d] * velb[d] * rinv;
  }
  Ub[0] += rhob;
#pragma unroll
  for (int d = 0; d < D; ++d) Ub[(1 + d) * ustride] += mb[d];
  Ub[(NV - 1) * ustride] += Eb;
}

__device__ __forceinline__ double dsign(double x) { return ipos(x) ? 1.0 : (ineg(x) ? -1.0 : 0.0); }

/* Reverse of face_flux_smem for one face.  Fb: adjoint of the face flux.  flags: the
   forward's NV x 2 flag bytes of this face (null: decided again here).  The adjoint of
   stencil point q, component v, is ADDED to Ub[(q * NV + v) * ustride]. */
template <int NV, int K, int LIM, int AXIS, int LANES>
__device__ __forceinline__ void face_vjp_smem(const double* sm, const double* rec, int NP, int jf, int lane,
                                              double gamma, const SchemeDev& sch, const uint8_t* flags,
                                              const double (&Fb)[NV], double* Ub, int ustride, int& st) {
  using L = PointLayout<NV>;
  constexpr int D = NV - 2;
  constexpr int H = K / 2;
  auto pidx = [&](int q) { return (jf + q) * LANES + lane; };
  auto P = [&](int comp, int q) -> double { return sm[comp * NP + pidx(q)]; };
  /* ---- forward quantities of the face ---- */
  const double sL = P(L::cS, H - 1), sR = P(L::cS, H);
  const double wsum = rcp_nr(sL + sR);
  double ut[D], q2 = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    ut[d] = (sL * P(L::cV + d, H - 1) + sR * P(L::cV + d, H)) * wsum;
    q2 += ut[d] * ut[d];
  }
  const double Ht = (sL * P(L::cH, H - 1) + sR * P(L::cH, H)) * wsum;
  const double c2 = (gamma - 1.0) * (Ht - 0.5 * q2);
  const double cinv = rsqrt_nr(c2);
  const double ct = c2 * cinv;
  const double b1 = (gamma - 1.0) * (cinv * cinv);
  const double b2 = 0.5 * q2 * b1;
  const double una = ut[AXIS];
  double a_m = 0.0, a_0 = 0.0, a_p = 0.0;
  int i_m = -1, i_0 = -1, i_p = -1;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const double xm = P(L::cLm, q), x0 = iabs(P(L::cV + AXIS, q)), xp = P(L::cLp, q);
    if (dbits(a_m) < dbits(xm)) { a_m = xm; i_m = q; }
    if (dbits(a_0) < dbits(x0)) { a_0 = x0; i_0 = q; }
    if (dbits(a_p) < dbits(xp)) { a_p = xp; i_p = q; }
  }
  /* ---- adjoint accumulators ---- */
  double utb[D];
#pragma unroll
  for (int d = 0; d < D; ++d) utb[d] = 0.0;
  double Htb = 0.0, ctb = 0.0, cinvb = 0.0, b1b = 0.0, b2b = 0.0, amb = 0.0, a0b = 0.0, apb = 0.0;
  double Fq[K][NV];
#pragma unroll
  for (int q = 0; q < K; ++q)
#pragma unroll
    for (int v = 0; v < NV; ++v) Fq[q][v] = 0.0;
  /* central combination of the point fluxes, for fields smooth on both sides */
  const unsigned full = (1u << (K - 2)) - 1u;
  const bool use_fc = sch.default_d;
  double Fc[NV], accS[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    accS[v] = 0.0;
    Fc[v] = 0.0;
    if (use_fc) {
      double arr[K];
#pragma unroll
      for (int q = 0; q < K; ++q) arr[q] = P(L::cF + v, q);
      Fc[v] = central_fn<K>(arr);
    }
  }

#pragma unroll 1
  for (int s = 0; s < NV; ++s) {
    const bool acoustic = (s == 0) || (s == NV - 1);
    const double sg = (s == 0) ? 1.0 : -1.0;
    const int dt = (s - 2) < AXIS ? (s - 2) : (s - 1);
    double utt = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) utt = (d == dt) ? ut[d] : utt;
    double l[NV];
    if (acoustic) {
      l[0] = 0.5 * (b2 + sg * una * cinv);
#pragma unroll
      for (int d = 0; d < D; ++d) l[1 + d] = 0.5 * (-b1 * ut[d] - (d == AXIS ? sg * cinv : 0.0));
      l[NV - 1] = 0.5 * b1;
    } else if (s == 1) {
      l[0] = 1.0 - b2;
#pragma unroll
      for (int d = 0; d < D; ++d) l[1 + d] = b1 * ut[d];
      l[NV - 1] = -b1;
    } else {
      l[0] = -utt;
#pragma unroll
      for (int d = 0; d < D; ++d) l[1 + d] = (d == dt) ? 1.0 : 0.0;
      l[NV - 1] = 0.0;
    }
    const double ha = 0.5 * ((s == 0) ? a_m : (s == NV - 1 ? a_p : a_0));
    /* both split sides smooth with the maximal-order weights: f+ + f- = sum_q c_q (g+_q + g-_q)
       = l . sum_q c_q F_q (the central coefficients are symmetric): no alpha, no W */
    const bool smooth_lane = flags && use_fc && ((flags[2 * s] & 63u) == full) && ((flags[2 * s + 1] & 63u) == full);
    /* one path per warp: the general path is exact for smooth fields too */
    const bool smooth = __all_sync(__activemask(), smooth_lane);
    double fs = 0.0;
    bool lin_central = smooth;
    double W[K], gp[K], vm[K], op[K], omm[K];
    if (smooth) {
#pragma unroll
      for (int v = 0; v < NV; ++v) fs = fma(l[v], Fc[v], fs);
    } else {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double w, g;
      if (acoustic || s == 1) {
        w = l[0] * P(L::cU, q);
        g = l[0] * P(L::cF, q);
#pragma unroll
        for (int v = 1; v < NV; ++v) {
          w = fma(l[v], P(L::cU + v, q), w);
          g = fma(l[v], P(L::cF + v, q), g);
        }
      } else {  /* the forward's sparse shear projection */
        w = fma(-utt, P(L::cU, q), P(L::cU + 1 + dt, q));
        g = fma(-utt, P(L::cF, q), P(L::cF + 1 + dt, q));
      }
      const double hg = 0.5 * g;
      W[q] = w;
      gp[q] = fma(ha, w, hg);
      vm[K - 1 - q] = fma(-ha, w, hg);
    }
    unsigned bp, bm;
    if (flags) {
      bp = flags[2 * s] & 63u;
      bm = flags[2 * s + 1] & 63u;
    } else {
      unsigned f1, f2;
      teno_m<K, LIM>(gp, sch, f1, st);
      teno_m<K, LIM>(vm, sch, f2, st);
      bp = f1 & 63u;
      bm = f2 & 63u;
    }
    const bool cp = teno_m_weights<K, LIM>(gp, bp, sch, op);
    const bool cm = teno_m_weights<K, LIM>(vm, bm, sch, omm);
#pragma unroll
    for (int q = 0; q < K; ++q) fs += op[q] * gp[q] + omm[q] * vm[q];
    /* both reconstructions are the central scheme: the cheap reverse applies */
    lin_central = use_fc && __all_sync(__activemask(), cp && cm);
    }
    /* back-projection F = sum_s r_s fs: adjoint of fs and of r_s */
    double fsb;
    if (acoustic) {
      const double sr = -sg;
      fsb = Fb[0];
#pragma unroll
      for (int d = 0; d < D; ++d) fsb += (ut[d] + (d == AXIS ? sr * ct : 0.0)) * Fb[1 + d];
      fsb += (Ht + sr * una * ct) * Fb[NV - 1];
#pragma unroll
      for (int d = 0; d < D; ++d) utb[d] += fs * Fb[1 + d];
      ctb += sr * fs * Fb[1 + AXIS] + sr * una * fs * Fb[NV - 1];
      Htb += fs * Fb[NV - 1];
      utb[AXIS] += sr * ct * fs * Fb[NV - 1];
    } else if (s == 1) {
      fsb = Fb[0];
#pragma unroll
      for (int d = 0; d < D; ++d) fsb += ut[d] * Fb[1 + d];
      fsb += 0.5 * q2 * Fb[NV - 1];
#pragma unroll
      for (int d = 0; d < D; ++d) utb[d] += fs * (Fb[1 + d] + ut[d] * Fb[NV - 1]);
    } else {
      fsb = utt * Fb[NV - 1];
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (d == dt) fsb += Fb[1 + d];
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (d == dt) utb[d] += fs * Fb[NV - 1];
    }
    double lb[NV];
    if (lin_central) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        lb[v] = fsb * Fc[v];
        accS[v] = fma(fsb, l[v], accS[v]);
      }
    } else {
      /* frozen reconstructions and LLF split: g+ = ha W + G/2, g- = -ha W + G/2 */
      double hab = 0.0;
#pragma unroll
      for (int v = 0; v < NV; ++v) lb[v] = 0.0;
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const double gpb = op[q] * fsb, gmb = omm[K - 1 - q] * fsb;
        const double Wb = ha * (gpb - gmb), Gb = 0.5 * (gpb + gmb);
        hab += W[q] * (gpb - gmb);
        if (acoustic || s == 1) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            Ub[(q * NV + v) * ustride] += Wb * l[v];
            Fq[q][v] += Gb * l[v];
            lb[v] += Wb * P(L::cU + v, q) + Gb * P(L::cF + v, q);
          }
        } else {
          /* shear wave, l = (-u_t, e_t, 0): only l[0] depends on the Roe state */
          Ub[(q * NV) * ustride] -= Wb * utt;
          Fq[q][0] -= Gb * utt;
#pragma unroll
          for (int d = 0; d < D; ++d)
            if (d == dt) {
              Ub[(q * NV + 1 + d) * ustride] += Wb;
              Fq[q][1 + d] += Gb;
            }
          lb[0] += Wb * P(L::cU, q) + Gb * P(L::cF, q);
        }
      }
      if (s == 0) amb += 0.5 * hab;
      else if (s == NV - 1) apb += 0.5 * hab;
      else a0b += 0.5 * hab;
    }
    /* left eigenvector -> Roe state */
    if (acoustic) {
      b2b += 0.5 * lb[0];
      utb[AXIS] += 0.5 * sg * cinv * lb[0];
      cinvb += 0.5 * sg * una * lb[0];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        b1b -= 0.5 * ut[d] * lb[1 + d];
        utb[d] -= 0.5 * b1 * lb[1 + d];
      }
      cinvb -= 0.5 * sg * lb[1 + AXIS];
      b1b += 0.5 * lb[NV - 1];
    } else if (s == 1) {
      b2b -= lb[0];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        b1b += ut[d] * lb[1 + d];
        utb[d] += b1 * lb[1 + d];
      }
      b1b -= lb[NV - 1];
    } else {
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (d == dt) utb[d] -= lb[0];
    }
  }
  if (use_fc) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double e[K];
#pragma unroll
      for (int i = 0; i < K; ++i) e[i] = (i == q) ? 1.0 : 0.0;
      const double cq = central_fn<K>(e);  /* the central coefficient of point q (a constant) */
#pragma unroll
      for (int v = 0; v < NV; ++v) Fq[q][v] = fma(cq, accS[v], Fq[q][v]);
    }
  }
  /* ---- Roe average -> the two states of the face ---- */
  double q2b = 0.5 * b1 * b2b;
  b1b += 0.5 * q2 * b2b;
  cinvb += 2.0 * (gamma - 1.0) * cinv * b1b;
  double c2b = cinv * ctb;
  cinvb += c2 * ctb;
  c2b -= 0.5 * cinv * cinv * cinv * cinvb;
  Htb += (gamma - 1.0) * c2b;
  q2b -= 0.5 * (gamma - 1.0) * c2b;
  double vLb[D], vRb[D];
  double sLb = 0.0, sRb = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double u_b = utb[d] + 2.0 * ut[d] * q2b;
    vLb[d] = sL * wsum * u_b;
    vRb[d] = sR * wsum * u_b;
    sLb += (P(L::cV + d, H - 1) - ut[d]) * wsum * u_b;
    sRb += (P(L::cV + d, H) - ut[d]) * wsum * u_b;
  }
  const double HLb = sL * wsum * Htb, HRb = sR * wsum * Htb;
  sLb += (P(L::cH, H - 1) - Ht) * wsum * Htb;
  sRb += (P(L::cH, H) - Ht) * wsum * Htb;
  /* ---- points: physical flux, LLF alpha (argmax frozen), Roe inputs ---- */
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double velb[D];
#pragma unroll
    for (int d = 0; d < D; ++d) velb[d] = (q == H - 1) ? vLb[d] : ((q == H) ? vRb[d] : 0.0);
    double cb = 0.0;
    const double un = P(L::cV + AXIS, q), cq = P(L::cC, q);
    if (q == i_m) {
      const double sgm = dsign(un - cq);
      velb[AXIS] += amb * sgm;
      cb -= amb * sgm;
    }
    if (q == i_0) velb[AXIS] += a0b * dsign(un);
    if (q == i_p) {
      const double sgp = dsign(un + cq);
      velb[AXIS] += apb * sgp;
      cb += apb * sgp;
    }
    const double Hb = (q == H - 1) ? HLb : ((q == H) ? HRb : 0.0);
    const double sb = (q == H - 1) ? sLb : ((q == H) ? sRb : 0.0);
    double Fqq[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Fqq[v] = Fq[q][v];
    point_vjp<NV, AXIS>(sm, rec, NP, pidx(q), gamma, Fqq, velb, cb, Hb, sb, Ub + (q * NV) * ustride, ustride);
  }
}

}  // namespace tenom
