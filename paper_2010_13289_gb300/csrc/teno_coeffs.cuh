/* Generated by paper_2010_13289_gb300/csrc/gen_coeffs.py (exact rationals). Do not edit. */
#pragma once

namespace tenom {

/* Candidate fluxes f_{k,i+1/2} (Table 1), c = index of f_i in v. */
template <int c> __device__ __forceinline__ double cand0(const double* v) { return (-0.16666666666666666) * v[c + -1] + (0.8333333333333334) * v[c + 0] + (0.3333333333333333) * v[c + 1]; }
template <int c> __device__ __forceinline__ double cand1(const double* v) { return (0.3333333333333333) * v[c + 0] + (0.8333333333333334) * v[c + 1] + (-0.16666666666666666) * v[c + 2]; }
template <int c> __device__ __forceinline__ double cand2(const double* v) { return (0.3333333333333333) * v[c + -2] + (-1.1666666666666667) * v[c + -1] + (1.8333333333333333) * v[c + 0]; }
template <int c> __device__ __forceinline__ double cand3(const double* v) { return (0.25) * v[c + 0] + (1.0833333333333333) * v[c + 1] + (-0.4166666666666667) * v[c + 2] + (0.08333333333333333) * v[c + 3]; }
template <int c> __device__ __forceinline__ double cand4(const double* v) { return (-0.25) * v[c + -3] + (1.0833333333333333) * v[c + -2] + (-1.9166666666666667) * v[c + -1] + (2.0833333333333335) * v[c + 0]; }
template <int c> __device__ __forceinline__ double cand5(const double* v) { return (0.2) * v[c + 0] + (1.2833333333333334) * v[c + 1] + (-0.7166666666666667) * v[c + 2] + (0.2833333333333333) * v[c + 3] + (-0.05) * v[c + 4]; }

/* Smoothness indicators as sums of squares of difference combinations;
   D[t] = v[t+1] - v[t], e = index in D of the stencil's first difference.  With ABS the
   coefficients are replaced by their magnitudes (evaluated on |D| this bounds the
   rounding error of the form).  T: double, or float for the certified cutoff filter. */
/* beta0: cells i-1..i+1 (ABS: the same form with |coefficients|, for error bounds) */
template <int e, bool ABS = false, class T = double>
__device__ __forceinline__ T beta0(const T* D) {
  const T t0 = D[e + 0] + T(ABS ? 0.625 : -0.625) * D[e + 1];
  const T t1 = D[e + 1];
  return T(1.3333333333333333) * (t0 * t0) + T(0.8125) * (t1 * t1);
}
/* beta1: cells i+0..i+2 (ABS: the same form with |coefficients|, for error bounds) */
template <int e, bool ABS = false, class T = double>
__device__ __forceinline__ T beta1(const T* D) {
  const T t0 = D[e + 0] + T(ABS ? 0.55 : -0.55) * D[e + 1];
  const T t1 = D[e + 1];
  return T(3.3333333333333335) * (t0 * t0) + T(0.325) * (t1 * t1);
}
/* beta2: cells i-2..i+0 (ABS: the same form with |coefficients|, for error bounds) */
template <int e, bool ABS = false, class T = double>
__device__ __forceinline__ T beta2(const T* D) {
  const T t0 = D[e + 0] + T(ABS ? 1.375 : -1.375) * D[e + 1];
  const T t1 = D[e + 1];
  return T(1.3333333333333333) * (t0 * t0) + T(0.8125) * (t1 * t1);
}
/* beta3: cells i+0..i+3 (ABS: the same form with |coefficients|, for error bounds) */
template <int e, bool ABS = false, class T = double>
__device__ __forceinline__ T beta3(const T* D) {
  const T t0 = D[e + 0] + T(ABS ? 1.2311343141907927 : -1.2311343141907927) * D[e + 1] + T(ABS ? 0.43996203132415757 : 0.43996203132415757) * D[e + 2];
  const T t1 = D[e + 1] + T(ABS ? 0.4912908701749207 : -0.4912908701749207) * D[e + 2];
  const T t2 = D[e + 2];
  return T(8.779166666666667) * (t0 * t0) + T(2.143489954121183) * (t1 * t1) + T(0.062446182990134574) * (t2 * t2);
}
/* beta4: cells i-3..i+0 (ABS: the same form with |coefficients|, for error bounds) */
template <int e, bool ABS = false, class T = double>
__device__ __forceinline__ T beta4(const T* D) {
  const T t0 = D[e + 0] + T(ABS ? 2.5484460694698354 : -2.5484460694698354) * D[e + 1] + T(ABS ? 1.6946983546617915 : 1.6946983546617915) * D[e + 2];
  const T t1 = D[e + 1] + T(ABS ? 1.4896519285042333 : -1.4896519285042333) * D[e + 2];
  const T t2 = D[e + 2];
  return T(2.279166666666667) * (t0 * t0) + T(0.647775746496039) * (t1 * t1) + T(0.7959391658827218) * (t2 * t2);
}
/* beta5: cells i+0..i+4 (ABS: the same form with |coefficients|, for error bounds) */
template <int e, bool ABS = false, class T = double>
__device__ __forceinline__ T beta5(const T* D) {
  const T t0 = D[e + 0] + T(ABS ? 2.009233862747642 : -2.009233862747642) * D[e + 1] + T(ABS ? 1.5065049389351175 : 1.5065049389351175) * D[e + 2] + T(ABS ? 0.3999749810040957 : -0.3999749810040957) * D[e + 3];
  const T t1 = D[e + 1] + T(ABS ? 1.0617477851335366 : -1.0617477851335366) * D[e + 2] + T(ABS ? 0.3258026595958473 : 0.3258026595958473) * D[e + 3];
  const T t2 = D[e + 2] + T(ABS ? 0.46990440443089404 : -0.46990440443089404) * D[e + 3];
  const T t3 = D[e + 3];
  return T(21.412301587301588) * (t0 * t0) + T(8.593809217415075) * (t1 * t1) + T(0.6680662245581286) * (t2 * t2) + T(0.010369149413408286) * (t3 * t3);
}
/* betaK6: cells i-2..i+3 (ABS: the same form with |coefficients|, for error bounds) */
template <int e, bool ABS = false, class T = double>
__device__ __forceinline__ T betaK6(const T* D) {
  const T t0 = D[e + 0] + T(ABS ? 3.3800293620919937 : -3.3800293620919937) * D[e + 1] + T(ABS ? 4.137755308541131 : 4.137755308541131) * D[e + 2] + T(ABS ? 2.2318538224071762 : -2.2318538224071762) * D[e + 3] + T(ABS ? 0.4518745009732172 : 0.4518745009732172) * D[e + 4];
  const T t1 = D[e + 1] + T(ABS ? 1.8788632502196132 : -1.8788632502196132) * D[e + 2] + T(ABS ? 1.2398246217680282 : 1.2398246217680282) * D[e + 3] + T(ABS ? 0.2835945203123665 : -0.2835945203123665) * D[e + 4];
  const T t2 = D[e + 2] + T(ABS ? 0.8641384480158466 : -0.8641384480158466) * D[e + 3] + T(ABS ? 0.22441845180562248 : 0.22441845180562248) * D[e + 4];
  const T t3 = D[e + 3] + T(ABS ? 0.3841978250666033 : -0.3841978250666033) * D[e + 4];
  const T t4 = D[e + 4];
  return T(2.2468501984126985) * (t0 * t0) + T(3.6320275079835525) * (t1 * t1) + T(4.213886137822353) * (t2 * t2) + T(1.0316113515772065) * (t3 * t3) + T(0.03897812227306876) * (t4 * t4);
}
/* betaK8: cells i-3..i+4 (ABS: the same form with |coefficients|, for error bounds) */
template <int e, bool ABS = false, class T = double>
__device__ __forceinline__ T betaK8(const T* D) {
  const T t0 = D[e + 0] + T(ABS ? 5.466604721584358 : -5.466604721584358) * D[e + 1] + T(ABS ? 12.198899858981697 : 12.198899858981697) * D[e + 2] + T(ABS ? 14.267281363132112 : -14.267281363132112) * D[e + 3] + T(ABS ? 9.277023273612551 : 9.277023273612551) * D[e + 4] + T(ABS ? 3.1943586508786703 : -3.1943586508786703) * D[e + 5] + T(ABS ? 0.4565830920349984 : 0.4565830920349984) * D[e + 6];
  const T t1 = D[e + 1] + T(ABS ? 3.9757147804614976 : -3.9757147804614976) * D[e + 2] + T(ABS ? 6.202960846287914 : 6.202960846287914) * D[e + 3] + T(ABS ? 4.82340042530116 : -4.82340042530116) * D[e + 4] + T(ABS ? 1.8806300789772517 : 1.8806300789772517) * D[e + 5] + T(ABS ? 0.2949600148071268 : -0.2949600148071268) * D[e + 6];
  const T t2 = D[e + 2] + T(ABS ? 2.443616554928916 : -2.443616554928916) * D[e + 3] + T(ABS ? 2.344713526117375 : 2.344713526117375) * D[e + 4] + T(ABS ? 1.034025932382635 : -1.034025932382635) * D[e + 5] + T(ABS ? 0.17556067198924424 : 0.17556067198924424) * D[e + 6];
  const T t3 = D[e + 3] + T(ABS ? 1.3190710438551487 : -1.3190710438551487) * D[e + 4] + T(ABS ? 0.6793536099802688 : 0.6793536099802688) * D[e + 5] + T(ABS ? 0.12660537168943978 : -0.12660537168943978) * D[e + 6];
  const T t4 = D[e + 4] + T(ABS ? 0.7736629951239468 : -0.7736629951239468) * D[e + 5] + T(ABS ? 0.17448591500286423 : 0.17448591500286423) * D[e + 6];
  const T t5 = D[e + 5] + T(ABS ? 0.3736837202946995 : -0.3736837202946995) * D[e + 6];
  const T t6 = D[e + 6];
  return T(2.234854870582735) * (t0 * t0) + T(3.6638884397833413) * (t1 * t1) + T(5.644238245592201) * (t2 * t2) + T(7.367729894004351) * (t3 * t3) + T(2.9756305436346877) * (t4 * t4) + T(0.26204645894217) * (t5 * t5) + T(0.00612798797104159) * (t6 * t6);
}

/* K-point central reconstruction sum_k d_k f_k (all candidates smooth), c = index of f_i */
template <int c> __device__ __forceinline__ double central6(const double* v) { return (0.016666666666666666) * v[c + -2] + (-0.13333333333333333) * v[c + -1] + (0.6166666666666667) * v[c + 0] + (0.6166666666666667) * v[c + 1] + (-0.13333333333333333) * v[c + 2] + (0.016666666666666666) * v[c + 3]; }
template <int c> __device__ __forceinline__ double central8(const double* v) { return (-0.0035714285714285713) * v[c + -3] + (0.034523809523809526) * v[c + -2] + (-0.16547619047619047) * v[c + -1] + (0.6345238095238095) * v[c + 0] + (0.6345238095238095) * v[c + 1] + (-0.16547619047619047) * v[c + 2] + (0.034523809523809526) * v[c + 3] + (-0.0035714285714285713) * v[c + 4]; }

/* maximal-order optimal weights d_k, K = 6 */
__device__ __forceinline__ double dopt6(int k) {
  switch (k) {
    case 0: return 0.45;  /* 9/20 */
    case 1: return 0.3;  /* 3/10 */
    case 2: return 0.05;  /* 1/20 */
    case 3: return 0.2;  /* 1/5 */
    default: return 0.0;
  }
}
/* maximal-order optimal weights d_k, K = 8 */
__device__ __forceinline__ double dopt8(int k) {
  switch (k) {
    case 0: return 0.42857142857142855;  /* 3/7 */
    case 1: return 0.2571428571428571;  /* 9/35 */
    case 2: return 0.05714285714285714;  /* 2/35 */
    case 3: return 0.17142857142857143;  /* 6/35 */
    case 4: return 0.014285714285714285;  /* 1/70 */
    case 5: return 0.07142857142857142;  /* 1/14 */
    default: return 0.0;
  }
}

}  // namespace tenom
