/* Decision statistics of the TENO-M reconstruction (Sections 2.3-3.3 of arXiv 2010.13289),
 * for logging, not for the solver: per split side (face x characteristic field x f+/f-)
 * the cutoff decisions delta_k of Eq. cut-off taken in FP64, how close each is to the
 * cutoff (|chi_k - C_T| <= 1e-10 C_T, i.e. |gamma_k - C_T sum gamma| <= 1e-10 C_T sum
 * gamma), whether the certified FP32 filter decided the side and agreed, the share of
 * nonsmooth candidates per k, the sides where the limiter runs (Eq. mp_flux) and the
 * candidates whose value it changed, and the adaptive exponent [beta] of TENO8A
 * (Eq. cut-off_adjust), with [beta] near an integer counted apart. */
#pragma once
#include "tenom_recon.cuh"

namespace tenom {

enum {
  SC_SIDES = 0,          /* split sides examined */
  SC_CERTIFIED = 1,      /* sides decided by the certified FP32 filter */
  SC_DISAGREE = 2,       /* certified sides whose FP64 decisions differ (rounding-decided) */
  SC_ALL_SMOOTH = 3,     /* sides with every candidate smooth (K-point central formula) */
  SC_NONSMOOTH_K = 4,    /* 4 .. 9: nonsmooth candidates k = 0 .. K-3 */
  SC_LIMITED_SIDES = 10, /* sides with at least one nonsmooth candidate (the limiter runs) */
  SC_CHANGED = 11,       /* nonsmooth candidates whose value the limiter changed */
  SC_NEAR_CUT = 12,      /* decisions with |chi_k - C_T| <= 1e-10 C_T */
  SC_NEAR_CUT_SIDES = 13,
  SC_CT_EXP = 14,        /* 14 .. 17: adaptive [beta] = 7, 8, 9, 10 */
  SC_NEAR_BETA = 18,     /* adaptive beta within 1e-10 of an integer */
  SC_NONFINITE = 19,     /* sides with a non-finite sum of gamma */
  SC_COUNT = 20
};

template <int K, int LIM>
__device__ __forceinline__ void side_stats(const double (&v)[K], const SchemeDev& S, unsigned (&cnt)[SC_COUNT]) {
  constexpr int c = K / 2 - 1;
  constexpr int nk = K - 2;
  constexpr unsigned all = (1u << nk) - 1u;
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
    const double x = fma(tau, rcp_nr1(bk[k] + 1e-40), 1.0);  /* as the solver's FP64 path */
    const double x3 = x * x * x;
    gk[k] = x3 * x3;
    sum += gk[k];
  }
  double CT = S.ct_const, beta = 0.0;
  int ex = 7;
  if (S.ct_mode == CT_ADAPTIVE) CT = adaptive_ct<c>(D, &ex, &beta);
  const double thr = CT * sum;
  unsigned bits = 0;
  int near = 0;
#pragma unroll
  for (int k = 0; k < nk; ++k) {
    if (!(gk[k] < thr)) bits |= 1u << k;
    if (fabs(gk[k] - thr) <= 1e-10 * thr) ++near;
  }
  cnt[SC_SIDES] += 1;
  if (!isfinite(sum)) cnt[SC_NONFINITE] += 1;
  unsigned fb = 0;
  int fe = 7;
  if (teno_decide_fast<K>(v, S, fb, fe)) {
    cnt[SC_CERTIFIED] += 1;
    if (fb != bits || (S.ct_mode == CT_ADAPTIVE && fe != ex)) cnt[SC_DISAGREE] += 1;
  }
  cnt[SC_NEAR_CUT] += near;
  cnt[SC_NEAR_CUT_SIDES] += near ? 1 : 0;
  if (S.ct_mode == CT_ADAPTIVE) {
    cnt[SC_CT_EXP + (ex - 7)] += 1;
    if (fabs(beta - rint(beta)) <= 1e-10) cnt[SC_NEAR_BETA] += 1;
  }
  if (bits == all) {
    cnt[SC_ALL_SMOOTH] += 1;
    return;
  }
  cnt[SC_LIMITED_SIDES] += 1;
  double fk[nk];
  fk[0] = cand0<c>(v);
  fk[1] = cand1<c>(v);
  fk[2] = cand2<c>(v);
  fk[3] = cand3<c>(v);
  if constexpr (K == 8) {
    fk[4] = cand4<c>(v);
    fk[5] = cand5<c>(v);
  }
  double fmin = 0.0, fmax = 0.0, fl = 0.0;
  if (S.weights == W_TENOM) {
    if constexpr (LIM == LIM_MP) mp_bounds<c>(v, S, fmin, fmax);
    else fl = (LIM == LIM_TVD5) ? tvd5_flux<c>(v) : va_flux<c>(v);
  }
#pragma unroll
  for (int k = 0; k < nk; ++k) {
    if (bits >> k & 1u) continue;
    cnt[SC_NONSMOOTH_K + k] += 1;
    if (S.weights != W_TENOM) continue;  /* classical TENO drops the candidate: no limiter */
    const double f = (LIM == LIM_MP) ? median3(fk[k], fmin, fmax) : fl;
    if (f != fk[k]) cnt[SC_CHANGED] += 1;
  }
}

}  // namespace tenom
