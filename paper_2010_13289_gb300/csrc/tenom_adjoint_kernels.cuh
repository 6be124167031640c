/* Adjoint face sweeps: Z += L_a'(U)^T w for one axis a, where L_a(U)_i = -(F_{i+1/2} -
 * F_{i-1/2})/dx_a.  The adjoint of face f is Fbar_f = (w_f - w_{f-1})/dx_a (cells outside the
 * grid contribute nothing).  Each CTA owns the same tile as the forward face kernel and
 * stages the same point quantities.
 *
 * adj_face_kernel: branches from the cutoff flags (or decided again); each face thread
 *   rebuilds its frozen linear reconstructions and writes its K x NV point adjoints to its
 *   own shared-memory slots, then each staged point gathers the slots of the faces that
 *   touch it and adds the sum to Z.
 * adj_lin_kernel: from the linearisation the record kernels wrote (field_queue_item in
 *   tenom_face_fwd.cuh gives the tape layout); see the comment above it.
 * Z is updated with atomics: halo points are shared with the neighbouring tiles and
 * boundary ghosts fold onto their cell. */
#pragma once
#include "tenom_adjoint.cuh"

namespace tenom {

struct AdjArgs {
  const double* U;       /* state the operator was applied to [NV][ncell] */
  const uint8_t* flags;  /* forward flags of this axis [nface][NV][2], or null */
  const double* lin;     /* recorded linearisation of this axis [NV][2K+2][nface] (adj_lin_kernel) */
  const double* P;       /* cell primitives of U [NV + 2][ncell] (velocity, p, H, c, sqrt rho), or null */
  const double* w;       /* cell adjoint [NV][ncell] */
  double* Z;             /* accumulated L'^T w [NV][ncell] */
  int* status;
  int n[3];
  int bc[3];
  long long ncell;
  long long nface;       /* faces of this axis */
  double dx;
  double gamma;
  SchemeDev sch;
};

/* Position of a face tile in the grid (the forward face kernel's tiling) and the cell of
   each of its staged points. */
template <int NV, int K, int AXIS>
struct AdjTileMap {
  using T = FaceTile<NV, K, AXIS>;
  int f0, x0, o1, o2;
  long long sy, sz, sa;
  __device__ explicit AdjTileMap(const AdjArgs& A) {
    x0 = 0;
    o1 = 0;
    if (AXIS == 0) {
      const int row = blockIdx.x;
      o1 = row % A.n[1];
      o2 = row / A.n[1];
    } else {
      x0 = blockIdx.x * 32;
      o2 = blockIdx.z;
    }
    f0 = blockIdx.y * T::FACES;
    sy = A.n[0];
    sz = (long long)A.n[0] * A.n[1];
    sa = (AXIS == 0) ? 1 : (AXIS == 1 ? sy : sz);
  }
  __device__ long long point_cell(const AdjArgs& A, int p) const {
    const int lane = (AXIS == 0) ? 0 : (p & 31);
    const int row = (AXIS == 0) ? p : (p >> 5);
    const int j = bc_wrap(f0 - T::H + row, A.n[AXIS], A.bc[AXIS]);
    long long base;
    if (AXIS == 0) base = sy * o1 + sz * o2;
    else {
      int x = x0 + lane;
      x = x < A.n[0] ? x : A.n[0] - 1;
      base = x + (AXIS == 1 ? sz * o2 : sy * o2);
    }
    return base + sa * j;
  }
  /* linear index of face f at lateral lane position xg (the flags / face buffer order) */
  __device__ long long face_index(const AdjArgs& A, int f, int xg) const {
    if (AXIS == 0) return f + (long long)(A.n[0] + 1) * (o1 + (long long)A.n[1] * o2);
    if (AXIS == 1) return xg + (long long)A.n[0] * (f + (long long)(A.n[1] + 1) * o2);
    return xg + (long long)A.n[0] * (o2 + (long long)A.n[1] * f);
  }
  /* cells f-1 and f along the axis share this lateral offset */
  __device__ long long lateral(int xg) const {
    if (AXIS == 0) return sy * o1 + sz * o2;
    return xg + (AXIS == 1 ? sz * o2 : sy * o2);
  }
};

/* Stage the tile's point quantities (as the forward) and the per-point reciprocals
   rec = (1/rho, 1/(2 c rho), 1/(2 sqrt rho)) used by point_vjp. */
template <int NV, int K, int AXIS>
__device__ __forceinline__ void adj_stage(const AdjArgs& A, const AdjTileMap<NV, K, AXIS>& M, double* sm, double* rec,
                                          int& st) {
  using T = FaceTile<NV, K, AXIS>;
  for (int p = threadIdx.x; p < T::NP; p += T::THREADS) {
    const long long cell = M.point_cell(A, p);
    double u[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) u[q] = __ldg(A.U + q * A.ncell + cell);
    if (A.P) {
      double vel[NV - 2];
#pragma unroll
      for (int d = 0; d < NV - 2; ++d) vel[d] = __ldg(A.P + d * A.ncell + cell);
      stage_point_from<NV, AXIS>(u, vel, __ldg(A.P + (NV - 2) * A.ncell + cell), __ldg(A.P + (NV - 1) * A.ncell + cell),
                                 __ldg(A.P + NV * A.ncell + cell), __ldg(A.P + (NV + 1) * A.ncell + cell), sm, T::NP,
                                 p);
    } else {
      stage_point<NV, AXIS>(u, A.gamma, sm, T::NP, p, st);
    }
    const double c = sm[PointLayout<NV>::cC * T::NP + p], sr = sm[PointLayout<NV>::cS * T::NP + p];
    rec[p] = rcp_nr(u[0]);
    rec[T::NP + p] = rcp_nr(2.0 * c * u[0]);
    rec[2 * T::NP + p] = rcp_nr(2.0 * sr);
  }
}

/* Fbar of face f: (w_f - w_{f-1}) / dx (cells outside the grid contribute nothing) */
template <int NV>
__device__ __forceinline__ void face_adjoint(const AdjArgs& A, long long lat, long long sa, int f, int na,
                                             double (&Fb)[NV]) {
  const double rdx = 1.0 / A.dx;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double wr = (f < na) ? A.w[v * A.ncell + lat + sa * f] : 0.0;
    const double wl = (f >= 1) ? A.w[v * A.ncell + lat + sa * (f - 1)] : 0.0;
    Fb[v] = (wr - wl) * rdx;
  }
}

template <int NV, int K, int AXIS>
struct AdjTile {
  using F = FaceTile<NV, K, AXIS>;
  /* point tile + per-point reciprocals (1/rho, 1/(2 c rho), 1/(2 sqrt rho)) + per-face slots */
  static constexpr size_t SMEM = F::SMEM + sizeof(double) * (3 * (size_t)F::NP + (size_t)K * NV * F::THREADS);
};

template <int NV, int K, int LIM, int AXIS>
__global__ void __launch_bounds__(FaceTile<NV, K, AXIS>::THREADS)
adj_face_kernel(const AdjArgs A) {
  using T = FaceTile<NV, K, AXIS>;
  constexpr int TH = T::THREADS;
  extern __shared__ double sm[];
  double* rec = sm + PointLayout<NV>::NC * T::NP;
  double* slots = rec + 3 * T::NP;
  const int tid = threadIdx.x;
  const int na = A.n[AXIS];
  const AdjTileMap<NV, K, AXIS> M(A);
  int st = 0;
  adj_stage<NV, K, AXIS>(A, M, sm, rec, st);
#pragma unroll
  for (int k = 0; k < K * NV; ++k) slots[k * TH + tid] = 0.0;
  __syncthreads();

  const int lane = (AXIS == 0) ? 0 : (tid & 31);
  const int jf = (AXIS == 0) ? tid : (tid >> 5);
  const int f = M.f0 + jf;
  const int xg = M.x0 + lane;
  if ((f <= na) && (AXIS == 0 || xg < A.n[0])) {
    double Fb[NV];
    face_adjoint<NV>(A, M.lateral(xg), M.sa, f, na, Fb);
    const uint8_t* fl = A.flags ? A.flags + M.face_index(A, f, xg) * NV * 2 : nullptr;
    face_vjp_smem<NV, K, LIM, AXIS, T::LANES>(sm, rec, T::NP, jf, lane, A.gamma, A.sch, fl, Fb, slots + tid, TH, st);
  }
  __syncthreads();
  /* gather: point p (row r, lane) is stencil point q = r - jf of face row jf */
  for (int p = tid; p < T::NP; p += TH) {
    const int lanep = (AXIS == 0) ? 0 : (p & 31);
    const int row = (AXIS == 0) ? p : (p >> 5);
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int jr = row - q;
      if (jr >= 0 && jr < T::FACES) {
        const int t = jr * T::LANES + lanep;
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += slots[(q * NV + v) * TH + t];
      }
    }
    const long long cell = M.point_cell(A, p);
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (acc[v] != 0.0) atomicAdd(A.Z + v * A.ncell + cell, acc[v]);
  }
  if (st) atomicOr(A.status, st);
}

/* ------------------------------------------------------------------------------------------
 * Adjoint sweep from the recorded linearisation.  Per characteristic field s the forward
 * recorded fs, omegaW, sigma_q, delta_q with fs = sum_q sigma_q G_q + (alpha_s/2) delta_q W_q
 * (W_q = l_s . U_q, G_q = l_s . F_q), so the reverse needs no reconstruction, limiter or
 * projection replay.  The left eigenvectors share two vectors,
 *   l_{u-c} = (a + b)/2,  l_{u+c} = (a - b)/2,  l_entropy = e_0 - a,  l_shear = e_t - u_t e_0,
 *   a = (b2, -b1 u, b1),  b = (u_n / c, -e_n / c, 0),
 * so the adjoints of every field at a stencil point combine into the coefficients of e_0, a,
 * b and e_t before they are expanded (one expansion per point instead of one per field).
 * Point adjoints are summed in shared memory per point, in K phases (in phase q every face
 * adds to its q-th point; the points of one phase are distinct), and the reverse of the
 * point quantities (point_vjp, which is linear in its adjoint inputs) runs once per point
 * instead of once per (face, point). */
template <int NV, int K, int AXIS>
struct AdjLinTile {
  using F = FaceTile<NV, K, AXIS>;
  static constexpr int D = NV - 2;
  static constexpr int NA = 2 * NV + 3;   /* per point: Ubar direct (NV), Fbar (NV), alpha adjoints (3) */
  static constexpr int NR = 2 * (D + 2);  /* per face: Roe-state adjoints of its two centre points */
  static constexpr size_t SMEM = F::SMEM + sizeof(double) * ((size_t)(3 + NA) * F::NP + (size_t)NR * F::THREADS);
};

template <int NV, int K, int AXIS>
__global__ void __launch_bounds__(FaceTile<NV, K, AXIS>::THREADS)
adj_lin_kernel(const AdjArgs A) {
  using T = FaceTile<NV, K, AXIS>;
  using L = PointLayout<NV>;
  using TL = AdjLinTile<NV, K, AXIS>;
  constexpr int H = T::H, D = NV - 2, TH = T::THREADS, NP = T::NP, LANES = T::LANES;
  constexpr int NA = TL::NA, NR = TL::NR, RS = 2 * K + 2;
  constexpr int aU = 0, aF = NV, aM = 2 * NV;  /* alpha adjoints: aM + 0 (u-c), 1 (u), 2 (u+c) */
  extern __shared__ double sm[];
  double* rec = sm + L::NC * NP;
  double* acc = rec + 3 * NP;
  double* roe = acc + NA * NP;
  const int tid = threadIdx.x;
  const int na = A.n[AXIS];
  const AdjTileMap<NV, K, AXIS> M(A);
  int st = 0;
  adj_stage<NV, K, AXIS>(A, M, sm, rec, st);
  for (int i = tid; i < NA * NP; i += TH) acc[i] = 0.0;
  __syncthreads();

  const int lane = (AXIS == 0) ? 0 : (tid & 31);
  const int jf = (AXIS == 0) ? tid : (tid >> 5);
  const int f = M.f0 + jf;
  const int xg = M.x0 + lane;
  const bool active = (f <= na) && (AXIS == 0 || xg < A.n[0]);
  auto P = [&](int comp, int q) -> double { return sm[comp * NP + (jf + q) * LANES + lane]; };
  const double gm1 = A.gamma - 1.0;
  const long long ls = A.nface;

  /* ---- face state (the forward's Roe average and LLF alpha with its argmax) ---- */
  double ut[D], nb1u[D], q2 = 0.0, Ht = 0.0, c2 = 0.0, cinv = 0.0, ct = 0.0, b1 = 0.0, b2 = 0.0;
  double sL = 0.0, sR = 0.0, wsum = 0.0;
  int im[3] = {-1, -1, -1};
  double kW[NV], kG[NV], utb[D], Htb = 0.0, ctb = 0.0, alb[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int d = 0; d < D; ++d) {
    ut[d] = 0.0;
    nb1u[d] = 0.0;
    utb[d] = 0.0;
  }
#pragma unroll
  for (int s = 0; s < NV; ++s) {
    kW[s] = 0.0;
    kG[s] = 0.0;
  }
  const double* lin = nullptr;
  if (active) {
    sL = P(L::cS, H - 1);
    sR = P(L::cS, H);
    wsum = rcp_nr(sL + sR);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      ut[d] = (sL * P(L::cV + d, H - 1) + sR * P(L::cV + d, H)) * wsum;
      q2 += ut[d] * ut[d];
    }
    Ht = (sL * P(L::cH, H - 1) + sR * P(L::cH, H)) * wsum;
    c2 = gm1 * (Ht - 0.5 * q2);
    cinv = rsqrt_nr(c2);
    ct = c2 * cinv;
    b1 = gm1 * (cinv * cinv);
    b2 = 0.5 * q2 * b1;
#pragma unroll
    for (int d = 0; d < D; ++d) nb1u[d] = -b1 * ut[d];
    double am[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const double x[3] = {P(L::cLm, q), iabs(P(L::cV + AXIS, q)), P(L::cLp, q)};
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (dbits(am[i]) < dbits(x[i])) {
          am[i] = x[i];
          im[i] = q;
        }
    }
    double Fb[NV];
    face_adjoint<NV>(A, M.lateral(xg), M.sa, f, na, Fb);
    lin = A.lin + M.face_index(A, f, xg);
    const double una = ut[AXIS];
    /* back-projection F = sum_s r_s fs: adjoints of fs (fsb) and of r_s */
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      const double fs = lin[(s * RS) * ls], wW = lin[(s * RS + 1) * ls];
      const bool acoustic = (s == 0) || (s == NV - 1);
      const int fam = (s == 0) ? 0 : (s == NV - 1 ? 2 : 1);
      double fsb;
      if (acoustic) {
        const double sr = (s == 0) ? -1.0 : 1.0;  /* r: -c for u-c, +c for u+c */
        fsb = Fb[0];
#pragma unroll
        for (int d = 0; d < D; ++d) fsb += (ut[d] + (d == AXIS ? sr * ct : 0.0)) * Fb[1 + d];
        fsb += (Ht + sr * una * ct) * Fb[NV - 1];
#pragma unroll
        for (int d = 0; d < D; ++d) utb[d] += fs * Fb[1 + d];
        ctb += sr * fs * (Fb[1 + AXIS] + una * Fb[NV - 1]);
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
        const int dt = (s - 2) < AXIS ? (s - 2) : (s - 1);
        fsb = ut[dt] * Fb[NV - 1] + Fb[1 + dt];
        utb[dt] += fs * Fb[NV - 1];
      }
      /* fs depends on alpha_s through (alpha_s / 2) sum_q delta_q W_q */
      alb[fam] += 0.5 * fsb * wW;
      const double hf = acoustic ? 0.5 : 1.0;  /* the 1/2 of l_{u-+c} = (a +- b)/2 */
      kG[s] = hf * fsb;
      kW[s] = kG[s] * (0.5 * am[fam]);
    }
  }

  /* ---- per stencil point: U and F adjoints in the basis (e_0, a, b, e_t), K phases ---- */
  double ab[NV], bb0 = 0.0, bb1 = 0.0, tb[D];
#pragma unroll
  for (int v = 0; v < NV; ++v) ab[v] = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) tb[d] = 0.0;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double ubd[NV], fqd[NV];
    if (active) {
      double cU[NV], cF[NV];
#pragma unroll
      for (int s = 0; s < NV; ++s) {
        cF[s] = kG[s] * lin[(s * RS + 2 + q) * ls];
        cU[s] = kW[s] * lin[(s * RS + 2 + K + q) * ls];
      }
      double AU = cU[0] + cU[NV - 1] - cU[1], BU = cU[0] - cU[NV - 1], RU = cU[1];
      double AF = cF[0] + cF[NV - 1] - cF[1], BF = cF[0] - cF[NV - 1], RF = cF[1];
#pragma unroll
      for (int s = 2; s < NV - 1; ++s) {
        const int dt = (s - 2) < AXIS ? (s - 2) : (s - 1);
        RU = fma(-ut[dt], cU[s], RU);
        RF = fma(-ut[dt], cF[s], RF);
      }
      const double b0v = ut[AXIS] * cinv;
      ubd[0] = fma(AU, b2, fma(BU, b0v, RU));
      fqd[0] = fma(AF, b2, fma(BF, b0v, RF));
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int s = d < AXIS ? d + 2 : d + 1;  /* shear field of tangential axis d */
        const double xu = (d == AXIS) ? -BU * cinv : cU[s];
        const double xf = (d == AXIS) ? -BF * cinv : cF[s];
        ubd[1 + d] = fma(AU, nb1u[d], xu);
        fqd[1 + d] = fma(AF, nb1u[d], xf);
      }
      ubd[NV - 1] = AU * b1;
      fqd[NV - 1] = AF * b1;
      /* adjoints of the eigenvector entries: a (all components), b (rho, m_n), -u_t */
#pragma unroll
      for (int v = 0; v < NV; ++v) ab[v] = fma(AU, P(L::cU + v, q), fma(AF, P(L::cF + v, q), ab[v]));
      bb0 = fma(BU, P(L::cU, q), fma(BF, P(L::cF, q), bb0));
      bb1 = fma(BU, P(L::cU + 1 + AXIS, q), fma(BF, P(L::cF + 1 + AXIS, q), bb1));
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (d == AXIS) continue;
        const int s = d < AXIS ? d + 2 : d + 1;
        tb[d] = fma(cU[s], P(L::cU, q), fma(cF[s], P(L::cF, q), tb[d]));
      }
    }
    __syncthreads();  /* the previous phase's additions to these points are complete */
    if (active) {
      const int pq = (jf + q) * LANES + lane;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        acc[(aU + v) * NP + pq] += ubd[v];
        acc[(aF + v) * NP + pq] += fqd[v];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (im[i] == q) acc[(aM + i) * NP + pq] += alb[i];
    }
  }

  /* ---- eigenvector adjoints -> Roe average -> the two centre points ---- */
  double rl[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) rl[k] = 0.0;
  if (active) {
    const double una = ut[AXIS];
    double b2b = ab[0], b1b = ab[NV - 1];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      b1b -= ut[d] * ab[1 + d];
      utb[d] -= b1 * ab[1 + d];
      if (d != AXIS) utb[d] -= tb[d];
    }
    utb[AXIS] += cinv * bb0;
    double cinvb = una * bb0 - bb1;
    double q2b = 0.5 * b1 * b2b;
    b1b += 0.5 * q2 * b2b;
    cinvb += 2.0 * gm1 * cinv * b1b;
    double c2b = cinv * ctb;
    cinvb += c2 * ctb;
    c2b -= 0.5 * cinv * cinv * cinv * cinvb;
    Htb += gm1 * c2b;
    q2b -= 0.5 * gm1 * c2b;
    double sLb = 0.0, sRb = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const double u_b = (utb[d] + 2.0 * ut[d] * q2b) * wsum;
      rl[d] = sL * u_b;
      rl[D + 2 + d] = sR * u_b;
      sLb += (P(L::cV + d, H - 1) - ut[d]) * u_b;
      sRb += (P(L::cV + d, H) - ut[d]) * u_b;
    }
    const double hb = Htb * wsum;
    rl[D] = sL * hb;
    rl[2 * D + 2] = sR * hb;
    rl[D + 1] = sLb + (P(L::cH, H - 1) - Ht) * hb;
    rl[2 * D + 3] = sRb + (P(L::cH, H) - Ht) * hb;
  }
#pragma unroll
  for (int k = 0; k < NR; ++k) roe[k * TH + tid] = rl[k];
  __syncthreads();

  /* ---- per point: gather, reverse of the point quantities, add to Z ---- */
  for (int p = tid; p < NP; p += TH) {
    const int lanep = (AXIS == 0) ? 0 : (p & 31);
    const int row = (AXIS == 0) ? p : (p >> 5);
    double ub[NV], Fq[NV], velb[D], Hb = 0.0, sb = 0.0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      ub[v] = acc[(aU + v) * NP + p];
      Fq[v] = acc[(aF + v) * NP + p];
    }
#pragma unroll
    for (int d = 0; d < D; ++d) velb[d] = 0.0;
    const int jl = row - (H - 1), jr = row - H;  /* faces whose left / right centre point this is */
    if (jl >= 0 && jl < T::FACES) {
      const int t = jl * LANES + lanep;
#pragma unroll
      for (int d = 0; d < D; ++d) velb[d] += roe[d * TH + t];
      Hb += roe[D * TH + t];
      sb += roe[(D + 1) * TH + t];
    }
    if (jr >= 0 && jr < T::FACES) {
      const int t = jr * LANES + lanep;
#pragma unroll
      for (int d = 0; d < D; ++d) velb[d] += roe[(D + 2 + d) * TH + t];
      Hb += roe[(2 * D + 2) * TH + t];
      sb += roe[(2 * D + 3) * TH + t];
    }
    /* alpha = max |lambda| with the argmax frozen: lambda = u_n - c, u_n, u_n + c */
    const double un = sm[(L::cV + AXIS) * NP + p], c = sm[L::cC * NP + p];
    const double xm = acc[aM * NP + p] * dsign(un - c), x0 = acc[(aM + 1) * NP + p] * dsign(un);
    const double xp = acc[(aM + 2) * NP + p] * dsign(un + c);
    velb[AXIS] += xm + x0 + xp;
    const double cb = xp - xm;
    point_vjp<NV, AXIS>(sm, rec, NP, p, A.gamma, Fq, velb, cb, Hb, sb, ub, 1);
    const long long cell = M.point_cell(A, p);
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (ub[v] != 0.0) atomicAdd(A.Z + v * A.ncell + cell, ub[v]);
  }
  if (st) atomicOr(A.status, st);
}

}  // namespace tenom
