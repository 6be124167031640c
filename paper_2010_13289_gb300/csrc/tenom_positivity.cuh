/* Per-face arithmetic of the positivity-preserving flux limiter (Section 4.4, which applies
   the limiter of Hu, Adams & Shu 2013), shared by the single-grid limiter kernel
   (tenom_abi.cu) and the batched stage kernel (tenom_batch_kernel.cuh).

   The stage update is the mean of the one-sided states U_L - mu F (cell left of the face)
   and U_R + mu F (cell right), mu = 2 dim dt/dx_a, over the 2 dim faces of a cell; the face
   flux F^H is pulled towards the local Lax-Friedrichs flux
   F^LF = (F(U_L) + F(U_R) - alpha (U_R - U_L))/2, alpha = max(|u_a| + c) of the two cells,
   until both one-sided states keep density (a linear function of the blend factor, solved
   exactly) and then pressure (concave in the state, so the chord bound is safe) at or above
   eps = min(1e-13, the value with F^LF).  A face whose factors are both 1 is left as it is. */
#pragma once
#include "tenom_fastmath.cuh"

namespace tenom {

template <int NV>
__device__ __forceinline__ double state_pressure(const double (&W)[NV], double gm1) {
  double m2 = 0.0;
#pragma unroll
  for (int d = 1; d < NV - 1; ++d) m2 += W[d] * W[d];
  return gm1 * (W[NV - 1] - 0.5 * m2 / W[0]);
}

/* Proof in FP32 that the one-sided state W = U + m F (m = -+mu, F the high-order flux) has
   density >= 2e-13 and rho p / (gamma - 1) = rho E - |m|^2/2 >= 2e-13 rho / (gamma - 1),
   i.e. p >= 2e-13.  Inputs are truncated to FP32 on the integer pipe (relative error
   < 2^-23; below the FP32 normal range, absolute error < 1.2e-38; NaN and overflow become
   infinities, which fail every test).  With M_v = |u_v| + |m f_v| + 1e-30, each FP32 w_v
   is within 3.1e-7 M_v of the exact W_v, and the FP32 pressure form within 5e-7 B of the
   exact one, B the sum of the magnitudes it is built from (below); demanding 1e-5 M_0 and
   1e-5 B of headroom (20 times those bounds) makes a true result a proof.  False means
   "not proven", not "fails". */
template <int NV>
__device__ __forceinline__ bool screen_fp32(const double (&U)[NV], const double (&F)[NV], float m, float gm1f) {
  float w[NV], M[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float a = f32_rz(U[v]), f = f32_rz(F[v]);
    w[v] = fmaf(m, f, a);
    M[v] = fabsf(a) + fabsf(m * f) + 1e-30f;
  }
  float m2 = 0.0f, Bm = 0.0f;
#pragma unroll
  for (int d = 1; d < NV - 1; ++d) {
    m2 = fmaf(w[d], w[d], m2);
    Bm = fmaf(M[d], fabsf(w[d]) + M[d], Bm);
  }
  const float pe = w[0] * w[NV - 1];
  const float rp = gm1f * (pe - 0.5f * m2);
  const float B = gm1f * (M[0] * (fabsf(w[NV - 1]) + M[NV - 1]) + M[NV - 1] * (fabsf(w[0]) + M[0]) + Bm +
                          fabsf(pe) + 0.5f * m2);
  return (w[0] - 1e-5f * M[0] >= 2.0001e-13f) && (rp - 1e-5f * B >= 2.0001e-13f * (w[0] + 1e-5f * M[0]));
}

/* The early exit in FP64 (division-free): both one-sided states made with F^H have density
   and pressure (tested as rho p against 2e-13 rho) at least 2e-13, twice the largest floor,
   so neither factor can fall below 1. */
template <int NV>
__device__ __forceinline__ bool exit_fp64(const double (&Ua)[NV], const double (&Ub)[NV], const double (&FH)[NV],
                                          double mu, double gm1) {
  double W0[NV], W1[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    W0[v] = Ua[v] - mu * FH[v];
    W1[v] = Ub[v] + mu * FH[v];
  }
  double m0 = 0.0, m1 = 0.0;
#pragma unroll
  for (int d = 1; d < NV - 1; ++d) {
    m0 += W0[d] * W0[d];
    m1 += W1[d] * W1[d];
  }
  return (W0[0] >= 2e-13) && (W1[0] >= 2e-13) && (gm1 * (W0[0] * W0[NV - 1] - 0.5 * m0) >= 2e-13 * W0[0]) &&
         (gm1 * (W1[0] * W1[NV - 1] - 0.5 * m1) >= 2e-13 * W1[0]);
}

/* The limiter proper at one face of axis AXIS: cells Us[0] | Us[1], high-order flux F,
   rewritten in place when a factor is below 1 (returns whether it was). */
template <int NV, int AXIS>
__device__ __forceinline__ bool limit_core(const double (&Us)[2][NV], double (&F)[NV], double mu, double gamma) {
  const double gm1 = gamma - 1.0;
  double Fc[2][NV], sp[2];
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const double rho = Us[sd][0];
    double vel[NV - 2], ke = 0.0;
#pragma unroll
    for (int d = 0; d < NV - 2; ++d) {
      vel[d] = Us[sd][1 + d] / rho;
      ke += Us[sd][1 + d] * vel[d];
    }
    const double p = gm1 * (Us[sd][NV - 1] - 0.5 * ke);
    const double un = vel[AXIS];
    Fc[sd][0] = Us[sd][1 + AXIS];
#pragma unroll
    for (int d = 0; d < NV - 2; ++d) Fc[sd][1 + d] = Us[sd][1 + d] * un + (d == AXIS ? p : 0.0);
    Fc[sd][NV - 1] = (Us[sd][NV - 1] + p) * un;
    sp[sd] = fabs(un) + sqrt(gamma * p / rho);
  }
  const double alpha = fmax(sp[0], sp[1]);
  double FLF[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) FLF[v] = 0.5 * (Fc[0][v] + Fc[1][v] - alpha * (Us[1][v] - Us[0][v]));
  /* density factor over both one-sided states (left loses F, right gains it) */
  double th = 1.0;
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const double m = sd ? mu : -mu;
    const double rlf = Us[sd][0] + m * FLF[0];
    const double rh = Us[sd][0] + m * F[0];
    const double eps = fmin(1e-13, rlf);
    if (rh < eps) th = fmin(th, (rlf - eps) / (rlf - rh));
  }
  double F1[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) F1[v] = (th == 1.0) ? F[v] : FLF[v] + th * (F[v] - FLF[v]);
  /* pressure factor on the density-limited flux */
  double tp = 1.0;
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const double m = sd ? mu : -mu;
    double Wlf[NV], W1[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Wlf[v] = Us[sd][v] + m * FLF[v];
      W1[v] = Us[sd][v] + m * F1[v];
    }
    const double plf = state_pressure<NV>(Wlf, gm1), p1 = state_pressure<NV>(W1, gm1);
    const double eps = fmin(1e-13, plf);
    if (p1 < eps) tp = fmin(tp, (plf - eps) / (plf - p1));
  }
  if (!(th < 1.0 || tp < 1.0)) return false;
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = (tp == 1.0) ? F1[v] : FLF[v] + tp * (F1[v] - FLF[v]);
  return true;
}

/* Whole per-face limiter on values in registers: FP32 proof of the early exit, the FP64
   test, then the limiter proper (muf, gm1f: mu and gamma - 1 truncated to FP32). */
template <int NV, int AXIS>
__device__ __forceinline__ void positivity_face(const double (&Ua)[NV], const double (&Ub)[NV], double (&F)[NV],
                                                double mu, double gamma, float muf, float gm1f) {
  if (screen_fp32<NV>(Ua, F, -muf, gm1f) && screen_fp32<NV>(Ub, F, muf, gm1f)) return;
  if (exit_fp64<NV>(Ua, Ub, F, mu, gamma - 1.0)) return;
  double Us[2][NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    Us[0][v] = Ua[v];
    Us[1][v] = Ub[v];
  }
  limit_core<NV, AXIS>(Us, F, mu, gamma);
}

}  // namespace tenom
