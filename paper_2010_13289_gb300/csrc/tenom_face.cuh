/* Fused characteristic face-flux kernel (Section 4 of arXiv 2010.13289: Roe-averaged
 * characteristic decomposition, Rusanov / local Lax-Friedrichs splitting, TENO-M per
 * characteristic field and split side, back-projection).
 *
 * One CTA owns a tile of consecutive faces along the sweep axis:
 *   axis x : 128 faces of one row, one thread per face (x is contiguous);
 *   axis y,z: 32 contiguous x-columns (lanes) x FT faces along the axis (warps).
 * Phase 1 stages the tile's points (faces + K-1 halo points, boundary condition applied
 * at load: periodic wrap or zero-gradient clamp) and computes every point quantity once
 * into shared memory: U, the physical flux F_a(U), velocity, total enthalpy H, sound
 * speed c and sqrt(rho).  Phase 2 computes each face flux exactly once and writes it to
 * the face buffer [nvar][nface_a]; the cell update (flux difference) reads it later, so
 * both neighbouring cells use the same face value.
 */
#pragma once
#include <cstdint>
#include "tenom_recon.cuh"
#include "tenom_linear.cuh"
#include "tenom_fastmath.cuh"

namespace tenom {

struct FaceArgs {
  const double* U;    /* [NV][ncell] */
  double* Fhat;       /* [NV][nface] */
  uint8_t* flags;     /* [nface][NV][2] or null */
  double* lin;        /* linearisation [NV][2K+2][nface] (record kernels only) */
  int* status;        /* sticky status word */
  int n[3];
  int bc[3];
  long long ncell;
  long long nface;
  double gamma;
  SchemeDev sch;
};

/* shared-memory layout of the staged point quantities: component c of point p at c * NP + p */
template <int NV>
struct PointLayout {
  static constexpr int NC = 3 * NV + 3;
  static constexpr int cU = 0, cF = NV, cV = 2 * NV, cH = 3 * NV - 2, cC = 3 * NV - 1, cS = 3 * NV;
  static constexpr int cLm = 3 * NV + 1, cLp = 3 * NV + 2;
};

constexpr int FX_FACES = 128;  /* faces per CTA, x sweeps */
constexpr int FT_FACES = 8;    /* faces per CTA along the axis, y/z sweeps (x 32 lanes) */

template <int NV, int K, int AXIS>
struct FaceTile {
  static constexpr int H = K / 2;
  static constexpr int NC = PointLayout<NV>::NC;
  static constexpr int LANES = (AXIS == 0) ? 1 : 32;
  static constexpr int FACES = (AXIS == 0) ? FX_FACES : FT_FACES;
  static constexpr int ROWS = FACES + K - 1;     /* points along the axis */
  static constexpr int NP = ROWS * LANES;        /* points per tile */
  static constexpr int THREADS = FACES * LANES;
  static constexpr size_t SMEM = sizeof(double) * NC * NP;
};

__device__ __forceinline__ int bc_wrap(int j, int n, int bc) {
  if (bc == 0) {
    j %= n;
    return j < 0 ? j + n : j;
  }
  return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

/* Point quantities of the Euler equations for sweep axis AXIS (computed once per point):
   U, the physical flux F_AXIS(U), velocity, H, c, sqrt(rho), |u_a - c|, |u_a + c|. */
template <int NV, int AXIS>
__device__ __forceinline__ void stage_point(const double (&u)[NV], double gamma, double* sm, int NP, int p, int& st) {
  using L = PointLayout<NV>;
  constexpr int D = NV - 2;
  const double rho = u[0];
  const double rinv = rcp_nr(rho);
  double vel[D], ke = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    vel[d] = u[1 + d] * rinv;
    ke += u[1 + d] * vel[d];
  }
  const double pr = (gamma - 1.0) * (u[NV - 1] - 0.5 * ke);
  const double c = sqrt(gamma * pr * rinv);
  const double Hh = (u[NV - 1] + pr) * rinv;
  if (!ipos(rho)) st |= ST_RHO;
  if (!ipos(pr)) st |= ST_P;
  const double un = vel[AXIS];
#pragma unroll
  for (int q = 0; q < NV; ++q) sm[(L::cU + q) * NP + p] = u[q];
  sm[(L::cF + 0) * NP + p] = u[0] * un;
#pragma unroll
  for (int d = 0; d < D; ++d) sm[(L::cF + 1 + d) * NP + p] = u[1 + d] * un + (d == AXIS ? pr : 0.0);
  sm[(L::cF + NV - 1) * NP + p] = (u[NV - 1] + pr) * un;
#pragma unroll
  for (int d = 0; d < D; ++d) sm[(L::cV + d) * NP + p] = vel[d];
  sm[L::cH * NP + p] = Hh;
  sm[L::cC * NP + p] = c;
  sm[L::cS * NP + p] = sqrt(rho);
  sm[L::cLm * NP + p] = iabs(un - c);
  sm[L::cLp * NP + p] = iabs(un + c);
}

/* Flux at the face whose K stencil points are shared-memory points (jf + q) * LANES + lane,
   q = 0..K-1, of a tile laid out by PointLayout<NV> with NP points per component:
   Roe average of points K/2-1 and K/2, characteristic projection, LLF split, TENO-M per
   field and side, back-projection.  flags (may be null) receives NV x 2 bytes.
   REC: also write the face's linearisation to lin[j * lstride], j = s * (2K + 2) + ...:
   per characteristic field s the reconstructed fs = f+ + f-, omegaW = sum_q delta_q W_q,
   sigma_q (K) and delta_q (K), where with the frozen linear weights op (f+) and om (f-, on
   the mirrored stencil) fs = sum_q sigma_q G_q + (alpha_s/2) delta_q W_q:
   sigma_q = (op_q + om_{K-1-q})/2, delta_q = op_q - om_{K-1-q}. */
template <int NV, int K, int LIM, int AXIS, int LANES, bool REC = false>
__device__ __forceinline__ void face_flux_smem(const double* sm, int NP, int jf, int lane, double gamma,
                                               const SchemeDev& sch, double (&Fh)[NV], uint8_t* flags, int& st,
                                               double* lin = nullptr, long long lstride = 0) {
  using L = PointLayout<NV>;
  constexpr int D = NV - 2;
  constexpr int H = K / 2;
  auto P = [&](int comp, int q) -> double {
    return sm[comp * NP + (jf + q) * LANES + lane];
  };
  /* Roe average of cells f-1 (point H-1) and f (point H) */
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
  if (!ipos(c2)) st |= ST_ROE;
  const double cinv = rsqrt_nr(c2);
  const double ct = c2 * cinv;
  const double b1 = (gamma - 1.0) * (cinv * cinv);
  const double b2 = 0.5 * q2 * b1;
  const double una = ut[AXIS];
  /* LLF: alpha_s = max over the K stencil points of |lambda_s|, one per eigenvalue family */
  double a_m = 0.0, a_0 = 0.0, a_p = 0.0;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    a_m = imax_nonneg(a_m, P(L::cLm, q));
    a_0 = imax_nonneg(a_0, iabs(P(L::cV + AXIS, q)));
    a_p = imax_nonneg(a_p, P(L::cLp, q));
  }

#pragma unroll
  for (int v = 0; v < NV; ++v) Fh[v] = 0.0;

#pragma unroll 1
  for (int s = 0; s < NV; ++s) {
    const bool acoustic = (s == 0) || (s == NV - 1);
    const double sg = (s == 0) ? 1.0 : -1.0;            /* l: +1 for u-c, -1 for u+c */
    const int dt = (s - 2) < AXIS ? (s - 2) : (s - 1);  /* shear fields: tangential axes in increasing order */
    double utt = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) utt = (d == dt) ? ut[d] : utt;
    /* left eigenvector l_s (closed form of R^{-1}) */
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
    /* characteristic projection of the K stencil points and LLF split
       g+- = (G +- alpha W)/2, evaluated as fma(+-alpha/2, W, G/2) */
    const double ha = 0.5 * ((s == 0) ? a_m : (s == NV - 1 ? a_p : a_0));
    double gp[K], gm[K], Wr[REC ? K : 1];
    if (acoustic || s == 1) {
#pragma unroll
      for (int q = 0; q < K; ++q) {
        double w = l[0] * P(L::cU, q), g = l[0] * P(L::cF, q);
#pragma unroll
        for (int v = 1; v < NV; ++v) {
          w = fma(l[v], P(L::cU + v, q), w);
          g = fma(l[v], P(L::cF + v, q), g);
        }
        const double hg = 0.5 * g;
        gp[q] = fma(ha, w, hg);
        gm[q] = fma(-ha, w, hg);
        if constexpr (REC) Wr[q] = w;
      }
    } else {
      /* shear wave: l = (-u_t, e_t, 0) */
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const double w = fma(-utt, P(L::cU, q), P(L::cU + 1 + dt, q));
        const double hg = 0.5 * fma(-utt, P(L::cF, q), P(L::cF + 1 + dt, q));
        gp[q] = fma(ha, w, hg);
        gm[q] = fma(-ha, w, hg);
        if constexpr (REC) Wr[q] = w;
      }
    }
    /* f+ on the upwind stencil, f- on the stencil mirrored about x_{i+1/2} */
    double vm[K];
#pragma unroll
    for (int q = 0; q < K; ++q) vm[q] = gm[K - 1 - q];
    unsigned flp, flm;
    double op[REC ? K : 1], om[REC ? K : 1];
    const double fplus = teno_m<K, LIM, REC>(gp, sch, flp, st, op);
    const double fminus = teno_m<K, LIM, REC>(vm, sch, flm, st, om);
    if (flags) {
      flags[s * 2 + 0] = (uint8_t)flp;
      flags[s * 2 + 1] = (uint8_t)flm;
    }
    const double fs = fplus + fminus;
    if constexpr (REC) {
      double* o = lin + (long long)s * (2 * K + 2) * lstride;
      double wW = 0.0;
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const double dq = op[q] - om[K - 1 - q];
        o[(2 + q) * lstride] = 0.5 * (op[q] + om[K - 1 - q]);
        o[(2 + K + q) * lstride] = dq;
        wW = fma(dq, Wr[q], wW);
      }
      o[0] = fs;
      o[lstride] = wW;
    }
    /* back-projection F += r_s fs */
    if (acoustic) {
      const double sr = -sg;                            /* r: -c for u-c, +c for u+c */
      Fh[0] += fs;
#pragma unroll
      for (int d = 0; d < D; ++d) Fh[1 + d] += (ut[d] + (d == AXIS ? sr * ct : 0.0)) * fs;
      Fh[NV - 1] += (Ht + sr * una * ct) * fs;
    } else if (s == 1) {
      Fh[0] += fs;
#pragma unroll
      for (int d = 0; d < D; ++d) Fh[1 + d] += ut[d] * fs;
      Fh[NV - 1] += 0.5 * q2 * fs;
    } else {
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (d == dt) Fh[1 + d] += fs;
      Fh[NV - 1] += utt * fs;
    }
  }
}

template <int NV, int K, int LIM, int AXIS, bool REC = false>
__global__ void __launch_bounds__(FaceTile<NV, K, AXIS>::THREADS)
face_kernel(const FaceArgs A) {
  using T = FaceTile<NV, K, AXIS>;
  constexpr int H = T::H;
  extern __shared__ double sm[];
  const int tid = threadIdx.x;

  /* --- tile coordinates --- */
  const int na = A.n[AXIS];
  int f0, x0 = 0, o1 = 0, o2 = 0;
  if (AXIS == 0) {
    const int row = blockIdx.x;          /* y + ny * z */
    o1 = row % A.n[1];
    o2 = row / A.n[1];
    f0 = blockIdx.y * T::FACES;
  } else {
    x0 = blockIdx.x * 32;
    f0 = blockIdx.y * T::FACES;
    o2 = blockIdx.z;                     /* AXIS 1: z ; AXIS 2: y */
  }
  const long long sx = 1, sy = A.n[0], sz = (long long)A.n[0] * A.n[1];
  const long long sa = (AXIS == 0) ? sx : (AXIS == 1 ? sy : sz);

  /* --- phase 1: point quantities --- */
  int st = 0;
  for (int p = tid; p < T::NP; p += T::THREADS) {
    const int lane = (AXIS == 0) ? 0 : (p & 31);
    const int row = (AXIS == 0) ? p : (p >> 5);
    const int j = bc_wrap(f0 - H + row, na, A.bc[AXIS]);
    long long base;
    if (AXIS == 0) base = sy * o1 + sz * o2;
    else {
      int x = x0 + lane;
      x = x < A.n[0] ? x : A.n[0] - 1;
      base = x + (AXIS == 1 ? sz * o2 : sy * o2);
    }
    const long long cell = base + sa * j;
    double u[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) u[q] = __ldg(A.U + q * A.ncell + cell);
    stage_point<NV, AXIS>(u, A.gamma, sm, T::NP, p, st);
  }
  __syncthreads();

  /* --- phase 2: one face per thread --- */
  const int lane = (AXIS == 0) ? 0 : (tid & 31);
  const int jf = (AXIS == 0) ? tid : (tid >> 5);
  const int f = f0 + jf;
  const int xg = x0 + lane;
  bool active = (f <= na) && (AXIS == 0 || xg < A.n[0]);
  if (active) {
    /* face linear index (n_a + 1 entries along the axis) */
    long long flin;
    if (AXIS == 0) flin = f + (long long)(A.n[0] + 1) * (o1 + (long long)A.n[1] * o2);
    else if (AXIS == 1) flin = xg + (long long)A.n[0] * (f + (long long)(A.n[1] + 1) * o2);
    else flin = xg + (long long)A.n[0] * (o2 + (long long)A.n[1] * f);
    double Fh[NV];
    face_flux_smem<NV, K, LIM, AXIS, T::LANES, REC>(sm, T::NP, jf, lane, A.gamma, A.sch, Fh,
                                                    A.flags ? A.flags + flin * NV * 2 : nullptr, st,
                                                    REC ? A.lin + flin : nullptr, A.nface);
#pragma unroll
    for (int v = 0; v < NV; ++v) A.Fhat[v * A.nface + flin] = Fh[v];
  }
  if (st) atomicOr(A.status, st);
}

}  // namespace tenom
