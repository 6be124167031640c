/* Fused characteristic face-flux kernel (Section 4 of arXiv 2010.13289: Roe-averaged
 * characteristic decomposition, Rusanov / local Lax-Friedrichs splitting, TENO-M per
 * characteristic field and split side, back-projection).
 *
 * One CTA owns a tile of consecutive faces along the sweep axis, one thread per face:
 *   axis x : a run of faces of one row (x is contiguous);
 *   axis y,z: contiguous x-columns (lanes) x faces along the axis.
 * (Tile sizes: FaceTile; forward and record kernels use fx_faces / FWD_LANES.)
 * Phase 1 stages the tile's points (faces + K-1 halo points, boundary condition applied
 * at load: periodic wrap or zero-gradient clamp) with every point quantity they need,
 * once, in shared memory (U, velocity, H, sqrt(rho), p, |u -+ c|; the forward and record
 * kernels add FP32 copies and differences for the screen, tenom_face_fwd.cuh).  Phase 2
 * computes each face flux exactly once and writes it to the face buffer [nvar][nface_a];
 * the cell update (flux difference) reads it later, so both neighbouring cells use the
 * same face value.
 */
#pragma once
#include <cstdint>
#include "tenom_recon.cuh"
#include "tenom_linear.cuh"
#include "tenom_stats.cuh"
#include "tenom_fastmath.cuh"
#include "tenom_face_fwd.cuh"

namespace tenom {

struct FaceArgs {
  const double* U;    /* [NV][ncell] */
  double* Fhat;       /* [NV][nface] */
  uint8_t* flags;     /* [nface][NV][2] or null */
  const double* P;    /* point primitives [NV + 2][ncell] (velocity, p, H, c, sqrt rho), or null */
  double* lin;        /* linearisation [NV][2K+2][nface] (record kernels only) */
  int* status;        /* sticky status word */
  unsigned long long* stats;  /* decision statistics [SC_COUNT] (statistics kernels only) */
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
/* threads (faces) per CTA of the forward and record kernels: 256 for K = 8 in 2D and 3D
   (one CTA queue over 8 warps, fewer halo points per face: x sweeps 256 faces of a row,
   y/z sweeps 16 x columns by 16 faces), 128 for K = 6 and for 1D grids (a short line is
   latency-bound: it runs faster spread over more, smaller CTAs) */
__host__ __device__ constexpr int fx_faces(int K, int NV) { return (K == 8 && NV > 3) ? 256 : 128; }
/* faces per CTA along the axis of the statistics kernels and the adjoint sweeps, y/z
   (x 32 lanes): 4, i.e. 128-thread CTAs */
__host__ __device__ constexpr int ft_faces(int K) { return (void)K, 4; }
/* forward and record kernels, y/z sweeps: FWD_LANES x columns by fx_faces(K, NV) / FWD_LANES
   faces (a warp takes two face rows): with K = 8 the tile stages 23 rows of 16 points for
   256 faces (1.4 staged points per face; 11 rows of 32 for 128 faces were 2.75) */
constexpr int FWD_LANES = 16;
/* resident threads per SM the forward and record kernels are compiled for: 512 (4 CTAs of
   128 threads or 2 of 256), 128 registers a thread (at most about 100 bytes of spills, at
   K = 8): the latency-bound kernel gains more from the fourth group of warps than it loses
   to the spills.  Statistics kernels: 3 CTAs of 128 threads, 168 registers. */
constexpr int FACE_THREADS_PER_SM = 512;
constexpr int FACE_CTAS_PER_SM_STATS = 3;

template <int NV, int K, int AXIS, bool FWDT = false>
struct FaceTile {
  static constexpr int H = K / 2;
  static constexpr int NC = PointLayout<NV>::NC;
  static constexpr int LANES = (AXIS == 0) ? 1 : (FWDT ? FWD_LANES : 32);
  static constexpr int FACES = (AXIS == 0) ? (FWDT ? fx_faces(K, NV) : FX_FACES) : (FWDT ? fx_faces(K, NV) / FWD_LANES : ft_faces(K));
  static constexpr int ROWS = FACES + K - 1;     /* points along the axis */
  static constexpr int NP = ROWS * LANES;        /* points per tile */
  static constexpr int THREADS = FACES * LANES;
  static constexpr size_t SMEM = sizeof(double) * NC * NP;
  /* forward and record kernels (FwdFace): their point layout, one field queue per warp,
     then the FP32 copies of the point data and the queue lengths */
  static constexpr int NCF = PointLayoutF<NV>::NC;
  static constexpr size_t FQDOUBLES = (size_t)(THREADS / 32) * FQCAP * fq_rows<NV>();
  static constexpr size_t SMEM_FWD = sizeof(double) * ((size_t)NCF * NP + FQDOUBLES) +
                                     sizeof(float) * (size_t)PointLayoutF<NV>::NF * NP + sizeof(int) * (THREADS / 32);
};

/* dynamic shared memory of face_kernel<..., REC, STATS> */
template <int NV, int K, int AXIS, bool REC, bool STATS>
constexpr size_t face_smem() {
  return !STATS ? FaceTile<NV, K, AXIS, true>::SMEM_FWD : FaceTile<NV, K, AXIS>::SMEM;
}

__device__ __forceinline__ int bc_wrap(int j, int n, int bc) {
  if (bc == 0) {
    j %= n;
    return j < 0 ? j + n : j;
  }
  return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

/* Primitive quantities of one point: velocity, pressure p = (gamma - 1)(E - rho|u|^2/2),
   total enthalpy H = (E + p)/rho, sound speed c = sqrt(gamma p / rho), sqrt(rho). */
template <int NV>
__device__ __forceinline__ void point_prims(const double (&u)[NV], double gamma, double (&vel)[NV - 2], double& pr,
                                            double& Hh, double& c, double& sr, int& st) {
  constexpr int D = NV - 2;
  const double rho = u[0];
  const double rinv = rcp_nr(rho);
  double ke = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    vel[d] = u[1 + d] * rinv;
    ke += u[1 + d] * vel[d];
  }
  pr = (gamma - 1.0) * (u[NV - 1] - 0.5 * ke);
  c = sqrt(gamma * pr * rinv);
  Hh = (u[NV - 1] + pr) * rinv;
  sr = sqrt(rho);
  if (!ipos(rho)) st |= ST_RHO;
  if (!ipos(pr)) st |= ST_P;
}

/* Point quantities of the Euler equations for sweep axis AXIS, written to the tile from U
   and its primitives: U, the physical flux F_AXIS(U), velocity, H, c, sqrt(rho),
   |u_a - c|, |u_a + c|. */
template <int NV, int AXIS>
__device__ __forceinline__ void stage_point_from(const double (&u)[NV], const double (&vel)[NV - 2], double pr,
                                                 double Hh, double c, double sr, double* sm, int NP, int p) {
  using L = PointLayout<NV>;
  constexpr int D = NV - 2;
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
  sm[L::cS * NP + p] = sr;
  sm[L::cLm * NP + p] = iabs(un - c);
  sm[L::cLp * NP + p] = iabs(un + c);
}

/* Point quantities computed here (once per point of the tile). */
template <int NV, int AXIS>
__device__ __forceinline__ void stage_point(const double (&u)[NV], double gamma, double* sm, int NP, int p, int& st) {
  double vel[NV - 2], pr, Hh, c, sr;
  point_prims<NV>(u, gamma, vel, pr, Hh, c, sr, st);
  stage_point_from<NV, AXIS>(u, vel, pr, Hh, c, sr, sm, NP, p);
}

/* Flux at the face whose K stencil points are shared-memory points (jf + q) * LANES + lane,
   q = 0..K-1, of a tile laid out by PointLayout<NV> with NP points per component:
   Roe average of points K/2-1 and K/2, characteristic projection, LLF split, TENO-M per
   field and side (each lane its own), back-projection.  flags (may be null) receives NV x 2
   bytes.  The batched stage kernel's face flux; STATS: the decision statistics of both
   sides of every field into cnt (SC_COUNT counters) instead of the flux. */
template <int NV, int K, int LIM, int AXIS, int LANES, bool STATS = false>
__device__ __forceinline__ void face_flux_smem(const double* sm, int NP, int jf, int lane, double gamma,
                                               const SchemeDev& sch, double (&Fh)[NV], uint8_t* flags, int& st,
                                               unsigned* cnt = nullptr) {
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
  /* back-projection F += r_s fs (right eigenvector of field s) */
  auto backproj = [&](int s, double fs) {
    if ((s == 0) || (s == NV - 1)) {
      const double sr = (s == 0) ? -1.0 : 1.0;         /* r: -c for u-c, +c for u+c */
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
      const int dt = (s - 2) < AXIS ? (s - 2) : (s - 1);
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (d == dt) {
          Fh[1 + d] += fs;
          Fh[NV - 1] += ut[d] * fs;
        }
    }
  };
  /* The acoustic pair and the entropy field share the vectors a = (b2, -b1 u, b1) and
     b = (u_n / c, -e_n / c, 0): l_{u-+c} = (a +- b)/2, l_0 = e_0 - a.  Per stencil point
     A = a.U/2, B = b.U/2, AF = a.F/4, BF = b.F/4 once, then W_{u-+c} = A +- B,
     G_{u-+c}/2 = AF +- BF, W_0 = rho - 2A, G_0/2 = F_rho/2 - 2AF. */
  double pA[K], pB[K], pAF[K], pBF[K];
  {
    double ah[NV], aq[NV];
    ah[0] = 0.5 * b2;
#pragma unroll
    for (int d = 0; d < D; ++d) ah[1 + d] = -0.5 * b1 * ut[d];
    ah[NV - 1] = 0.5 * b1;
#pragma unroll
    for (int v = 0; v < NV; ++v) aq[v] = 0.5 * ah[v];
    const double bh0 = 0.5 * una * cinv, bh1 = -0.5 * cinv;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double a = ah[0] * P(L::cU, q), af = aq[0] * P(L::cF, q);
#pragma unroll
      for (int v = 1; v < NV; ++v) {
        a = fma(ah[v], P(L::cU + v, q), a);
        af = fma(aq[v], P(L::cF + v, q), af);
      }
      pA[q] = a;
      pAF[q] = af;
      pB[q] = fma(bh1, P(L::cU + 1 + AXIS, q), bh0 * P(L::cU, q));
      pBF[q] = 0.5 * fma(bh1, P(L::cF + 1 + AXIS, q), bh0 * P(L::cF, q));
    }
  }

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
    double gp[K], gm[K];
    if (acoustic) {
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const double w = fma(sg, pB[q], pA[q]), hg = fma(sg, pBF[q], pAF[q]);
        gp[q] = fma(ha, w, hg);
        gm[q] = fma(-ha, w, hg);
      }
    } else if (s == 1) {
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const double w = fma(-2.0, pA[q], P(L::cU, q)), hg = fma(-2.0, pAF[q], 0.5 * P(L::cF, q));
        gp[q] = fma(ha, w, hg);
        gm[q] = fma(-ha, w, hg);
      }
    } else {
      /* shear wave: l = (-u_t, e_t, 0) */
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const double w = fma(-utt, P(L::cU, q), P(L::cU + 1 + dt, q));
        const double hg = 0.5 * fma(-utt, P(L::cF, q), P(L::cF + 1 + dt, q));
        gp[q] = fma(ha, w, hg);
        gm[q] = fma(-ha, w, hg);
      }
    }
    /* f+ on the upwind stencil, f- on the stencil mirrored about x_{i+1/2} */
    double vm[K];
#pragma unroll
    for (int q = 0; q < K; ++q) vm[q] = gm[K - 1 - q];
    if constexpr (STATS) {  /* statistics of both sides' decisions instead of the flux */
      side_stats<K, LIM>(gp, sch, *reinterpret_cast<unsigned(*)[SC_COUNT]>(cnt));
      side_stats<K, LIM>(vm, sch, *reinterpret_cast<unsigned(*)[SC_COUNT]>(cnt));
      continue;
    }
    unsigned flp, flm;
    const double fplus = teno_m<K, LIM>(gp, sch, flp, st);
    const double fminus = teno_m<K, LIM>(vm, sch, flm, st);
    if (flags) {
      flags[s * 2 + 0] = (uint8_t)flp;
      flags[s * 2 + 1] = (uint8_t)flm;
    }
    backproj(s, fplus + fminus);
  }
}

template <int NV, int K, int LIM, int AXIS, bool REC = false, bool STATS = false>
__global__ void __launch_bounds__(FaceTile<NV, K, AXIS, !STATS>::THREADS,
                                  STATS ? FACE_CTAS_PER_SM_STATS : FACE_THREADS_PER_SM / FaceTile<NV, K, AXIS, !STATS>::THREADS)
face_kernel(const FaceArgs A) {
  using T = FaceTile<NV, K, AXIS, !STATS>;
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
    x0 = blockIdx.x * T::LANES;
    f0 = blockIdx.y * T::FACES;
    o2 = blockIdx.z;                     /* AXIS 1: z ; AXIS 2: y */
  }
  const long long sx = 1, sy = A.n[0], sz = (long long)A.n[0] * A.n[1];
  const long long sa = (AXIS == 0) ? sx : (AXIS == 1 ? sy : sz);

  /* --- phase 1: point quantities --- */
  constexpr bool FWD = !STATS;  /* forward and record kernels: the screened face flux */
  float* smf = reinterpret_cast<float*>(sm + (size_t)T::NCF * T::NP + T::FQDOUBLES);  /* forward kernels */
  int st = 0;
  for (int p = tid; p < T::NP; p += T::THREADS) {
    const int lane = (AXIS == 0) ? 0 : (p % T::LANES);
    const int row = (AXIS == 0) ? p : (p / T::LANES);
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
    if constexpr (FWD) {
      double vel[NV - 2], pr, Hh, cs, sr;
      if (A.P) {  /* primitives computed once per cell per stage (prim_kernel) */
#pragma unroll
        for (int d = 0; d < NV - 2; ++d) vel[d] = __ldg(A.P + d * A.ncell + cell);
        pr = __ldg(A.P + (NV - 2) * A.ncell + cell);
        Hh = __ldg(A.P + (NV - 1) * A.ncell + cell);
        cs = __ldg(A.P + NV * A.ncell + cell);
        sr = __ldg(A.P + (NV + 1) * A.ncell + cell);
      } else {
        point_prims<NV>(u, A.gamma, vel, pr, Hh, cs, sr, st);
      }
      stage_point_fwd<NV, AXIS>(u, vel, pr, Hh, cs, sr, sm, smf, T::NP, p);
    } else if (A.P) {  /* primitives computed once per cell per stage (prim_kernel) */
      double vel[NV - 2];
#pragma unroll
      for (int d = 0; d < NV - 2; ++d) vel[d] = __ldg(A.P + d * A.ncell + cell);
      stage_point_from<NV, AXIS>(u, vel, __ldg(A.P + (NV - 2) * A.ncell + cell), __ldg(A.P + (NV - 1) * A.ncell + cell),
                                 __ldg(A.P + NV * A.ncell + cell), __ldg(A.P + (NV + 1) * A.ncell + cell), sm, T::NP,
                                 p);
    } else {
      stage_point<NV, AXIS>(u, A.gamma, sm, T::NP, p, st);
    }
  }
  __syncthreads();
  int* wq_n = reinterpret_cast<int*>(smf + (size_t)PointLayoutF<NV>::NF * T::NP);  /* forward: queue lengths */
  if constexpr (FWD) {  /* differences to the next point along the axis, for the screen */
    for (int p = tid; p < T::NP - T::LANES; p += T::THREADS) stage_differences_fwd<NV, AXIS>(sm, smf, T::NP, p, p + T::LANES);
    __syncthreads();
  }

  /* --- phase 2: one face per thread --- */
  const int lane = (AXIS == 0) ? 0 : (tid % T::LANES);
  const int jf = (AXIS == 0) ? tid : (tid / T::LANES);
  const int f = f0 + jf;
  const int xg = x0 + lane;
  /* forward kernels on a periodic axis compute faces 0 .. n-1 only: face n has the same
     stencil points as face 0, and face 0's lanes write it to both places (face_grid sizes
     those launches for n faces, which drops the nearly empty last tile of every line) */
  const bool wrapped = FWD && A.bc[AXIS] == 0;
  bool active = (wrapped ? f < na : f <= na) && (AXIS == 0 || xg < A.n[0]);
  const unsigned am = __ballot_sync(0xffffffffu, active);  /* the lanes sharing the warp's queue */
  unsigned cnt[STATS ? SC_COUNT : 1];
#pragma unroll
  for (int q = 0; q < (STATS ? SC_COUNT : 1); ++q) cnt[q] = 0u;
  double Fh[NV];
  /* face linear index (n_a + 1 entries along the axis) */
  long long flin = 0;
  if (AXIS == 0) flin = f + (long long)(A.n[0] + 1) * (o1 + (long long)A.n[1] * o2);
  else if (AXIS == 1) flin = xg + (long long)A.n[0] * (f + (long long)(A.n[1] + 1) * o2);
  else flin = xg + (long long)A.n[0] * (o2 + (long long)A.n[1] * f);
  uint8_t* const flg = (active && A.flags) ? A.flags + flin * NV * 2 : nullptr;
  if constexpr (FWD) {
    /* screen every field, queue the rest; the CTA works through the queues together (more
       than one round only when a warp's queue fills) */
    constexpr int W = T::THREADS / 32;
    double* const fq0 = sm + (size_t)T::NCF * T::NP;
    double* const fq = fq0 + (size_t)(tid >> 5) * FQCAP * fq_rows<NV>();
    FwdFace<NV, K, LIM, AXIS, T::LANES, REC> F;
    if (active) F.begin(sm, T::NP, jf, lane, A.gamma, st);
    /* record kernels: the tape row of the face in tile row r, x column x0 + c */
    auto tape = [&](int r, int c) -> double* {
      const long long fr = f0 + r, xr = x0 + c;
      if (AXIS == 0) return A.lin + fr + (long long)(A.n[0] + 1) * (o1 + (long long)A.n[1] * o2);
      if (AXIS == 1) return A.lin + xr + (long long)A.n[0] * (fr + (long long)(A.n[1] + 1) * o2);
      return A.lin + xr + (long long)A.n[0] * (o2 + (long long)A.n[1] * fr);
    };
    const int rot = (int)((blockIdx.x + blockIdx.y + blockIdx.z) % W);
    bool again = true;
#pragma unroll 1
    while (again) {
      bool stopped = false;
      int mine = 0;
      if (active && F.s_next < NV) {
        stopped = !F.fields(smf, T::NP, jf, lane, A.sch, flg, fq, am, REC ? A.lin + flin : nullptr, A.nface);
        mine = F.nq;
      }
      const int wn = __reduce_max_sync(0xffffffffu, mine);
      if ((tid & 31) == 0) wq_n[tid >> 5] = wn;
      __syncthreads();
      field_queue_cta<NV, K, LIM, AXIS, T::LANES, T::THREADS, REC>(sm, T::NP, fq0, wq_n, A.sch, st, rot, tape,
                                                                   A.nface);
      again = __syncthreads_or(stopped);
      if (active) F.readback(fq, flg, A.sch);
    }
    if (active) F.finish(Fh);
  }
  if (active) {
    if constexpr (!FWD)
      face_flux_smem<NV, K, LIM, AXIS, T::LANES, STATS>(sm, T::NP, jf, lane, A.gamma, A.sch, Fh, flg, st, cnt);
    if constexpr (!STATS) {
#pragma unroll
      for (int v = 0; v < NV; ++v) A.Fhat[v * A.nface + flin] = Fh[v];
      if (wrapped && f == 0) {  /* face n of the line */
        long long fn;
        if (AXIS == 0) fn = na + (long long)(A.n[0] + 1) * (o1 + (long long)A.n[1] * o2);
        else if (AXIS == 1) fn = xg + (long long)A.n[0] * (na + (long long)(A.n[1] + 1) * o2);
        else fn = xg + (long long)A.n[0] * (o2 + (long long)A.n[1] * na);
#pragma unroll
        for (int v = 0; v < NV; ++v) A.Fhat[v * A.nface + fn] = Fh[v];
        if (A.flags) {
#pragma unroll
          for (int e = 0; e < 2 * NV; ++e) A.flags[fn * NV * 2 + e] = A.flags[flin * NV * 2 + e];
        }
        if constexpr (REC) {  /* the tape rows, complete after the last queue round's barrier */
#pragma unroll 1
          for (int r = 0; r < NV * (2 * K + 2); ++r) A.lin[r * A.nface + fn] = A.lin[r * A.nface + flin];
        }
      }
    }
  }
  if constexpr (STATS) {  /* warp sums, one 64-bit atomic per counter and warp */
#pragma unroll
    for (int q = 0; q < SC_COUNT; ++q) {
      const unsigned w = __reduce_add_sync(0xffffffffu, cnt[q]);
      if ((tid & 31) == 0 && w) atomicAdd(A.stats + q, (unsigned long long)w);
    }
  }
  if (st) atomicOr(A.status, st);
}

}  // namespace tenom
