/* Adjoint face sweep: Z += L_a'(U)^T w for one axis a, where L_a(U)_i = -(F_{i+1/2} -
 * F_{i-1/2})/dx_a.  The adjoint of face f is Fbar_f = (w_f - w_{f-1})/dx_a (cells outside the
 * grid contribute nothing).  Each CTA owns the same tile as the forward face kernel; every
 * face thread writes its K x NV point adjoints to its own shared-memory slots, then each
 * staged point gathers the slots of the faces that touch it and adds the sum to Z (atomic:
 * halo points are shared with the neighbouring tiles; boundary ghosts fold onto their cell). */
#pragma once
#include "tenom_adjoint.cuh"

namespace tenom {

struct AdjArgs {
  const double* U;       /* state the operator was applied to [NV][ncell] */
  const uint8_t* flags;  /* forward flags of this axis [nface][NV][2], or null */
  const double* w;       /* cell adjoint [NV][ncell] */
  double* Z;             /* accumulated L'^T w [NV][ncell] */
  int* status;
  int n[3];
  int bc[3];
  long long ncell;
  double dx;
  double gamma;
  SchemeDev sch;
};

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
  constexpr int H = T::H;
  constexpr int TH = T::THREADS;
  extern __shared__ double sm[];
  double* rec = sm + PointLayout<NV>::NC * T::NP;
  double* slots = rec + 3 * T::NP;
  const int tid = threadIdx.x;
  const int na = A.n[AXIS];
  int f0, x0 = 0, o1 = 0, o2 = 0;
  if (AXIS == 0) {
    const int row = blockIdx.x;
    o1 = row % A.n[1];
    o2 = row / A.n[1];
    f0 = blockIdx.y * T::FACES;
  } else {
    x0 = blockIdx.x * 32;
    f0 = blockIdx.y * T::FACES;
    o2 = blockIdx.z;
  }
  const long long sy = A.n[0], sz = (long long)A.n[0] * A.n[1];
  const long long sa = (AXIS == 0) ? 1 : (AXIS == 1 ? sy : sz);
  auto point_cell = [&](int p) -> long long {
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
    return base + sa * j;
  };
  int st = 0;
  for (int p = tid; p < T::NP; p += TH) {
    const long long cell = point_cell(p);
    double u[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) u[q] = __ldg(A.U + q * A.ncell + cell);
    stage_point<NV, AXIS>(u, A.gamma, sm, T::NP, p, st);
    const double c = sm[PointLayout<NV>::cC * T::NP + p], sr = sm[PointLayout<NV>::cS * T::NP + p];
    rec[p] = rcp_nr(u[0]);
    rec[T::NP + p] = rcp_nr(2.0 * c * u[0]);
    rec[2 * T::NP + p] = rcp_nr(2.0 * sr);
  }
#pragma unroll
  for (int k = 0; k < K * NV; ++k) slots[k * TH + tid] = 0.0;
  __syncthreads();

  const int lane = (AXIS == 0) ? 0 : (tid & 31);
  const int jf = (AXIS == 0) ? tid : (tid >> 5);
  const int f = f0 + jf;
  const int xg = x0 + lane;
  if ((f <= na) && (AXIS == 0 || xg < A.n[0])) {
    /* cells f-1 and f along the axis at this lateral position */
    long long lat;
    if (AXIS == 0) lat = sy * o1 + sz * o2;
    else lat = xg + (AXIS == 1 ? sz * o2 : sy * o2);
    double Fb[NV];
    const double rdx = 1.0 / A.dx;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double wr = (f < na) ? A.w[v * A.ncell + lat + sa * f] : 0.0;
      const double wl = (f >= 1) ? A.w[v * A.ncell + lat + sa * (f - 1)] : 0.0;
      Fb[v] = (wr - wl) * rdx;
    }
    const uint8_t* fl = nullptr;
    if (A.flags) {
      long long flin;
      if (AXIS == 0) flin = f + (long long)(A.n[0] + 1) * (o1 + (long long)A.n[1] * o2);
      else if (AXIS == 1) flin = xg + (long long)A.n[0] * (f + (long long)(A.n[1] + 1) * o2);
      else flin = xg + (long long)A.n[0] * (o2 + (long long)A.n[1] * f);
      fl = A.flags + flin * NV * 2;
    }
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
    const long long cell = point_cell(p);
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (acc[v] != 0.0) atomicAdd(A.Z + v * A.ncell + cell, acc[v]);
  }
  if (st) atomicOr(A.status, st);
}

}  // namespace tenom
