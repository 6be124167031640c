/* Host side of the C ABI declared in include/tenom.h, plus the element-wise kernels:
 * primitive -> conserved state, cell update (flux difference + SSP-RK3 stage combine),
 * CFL reduction and the FP64 throughput probe.  The face kernels live in
 * tenom_face_nv{3,4,5}.cu. */
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tenom.h"
#include "tenom_internal.h"
#include "tenom_adjoint_kernels.cuh"
#include "tenom_positivity.cuh"

namespace tenom {

/* ---------------------------------------------------------------- kernels */

/* U = (rho, rho u, p/(gamma-1) + rho|u|^2/2) from (rho, u, p). */
template <int NV>
__global__ void init_state_kernel(const double* __restrict__ prim, double* __restrict__ U, long long nc,
                                  double gamma) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x) {
    const double rho = prim[c];
    double ke = 0.0;
#pragma unroll
    for (int d = 0; d < NV - 2; ++d) {
      const double u = prim[(1 + d) * nc + c];
      U[(1 + d) * nc + c] = rho * u;
      ke += rho * u * u;
    }
    U[c] = rho;
    U[(NV - 1) * nc + c] = prim[(NV - 1) * nc + c] / (gamma - 1.0) + 0.5 * ke;
  }
}

/* Flux difference -sum_a (F_{a,i+1/2} - F_{a,i-1/2}) / dx_a (Eq. approximateEq) and the
   SSP-RK3 stage combine of one cell: mode 0 out = L (operator), 1 out = Us + dt L (stage
   1), 2 out = cA U0 + cB (Us + dt L) (stages 2, 3); dt = 0 (a step past t_end) keeps Us. */
struct CellUpdate {
  const double* F[3];  /* face buffers per axis [NV][nface_a] */
  const double* U0;    /* U^n (stages 2, 3) */
  const double* Us;    /* stage input state */
  double* out;         /* stage output or dU/dt */
  const double* dt;    /* device dt (null for the operator) */
  double rdx[3];       /* 1 / dx_a */
  long long nface[3];
  double cA, cB;
  int mode;
};

/* the cell update of cell c whose x-face difference F_{x,i+1/2} - F_{x,i-1/2} is dfx; the
   other axes' faces at fl[a] and fl[a] + fs[a] */
template <int NV>
__device__ __forceinline__ void cell_update(const CellUpdate& A, long long nc, long long c, const double (&dfx)[NV],
                                            const long long (&fl)[3], const long long (&fs)[3], double dt) {
  constexpr int DIM = NV - 2;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double r = 0.0;
    r = r - dfx[v] * A.rdx[0];
#pragma unroll
    for (int a = 1; a < DIM; ++a) {
      const double* F = A.F[a] + v * A.nface[a];
      r = r - (F[fl[a] + fs[a]] - F[fl[a]]) * A.rdx[a];
    }
    if (A.mode == 0) {
      A.out[v * nc + c] = r;
    } else if (dt == 0.0) {
      /* a step past t_end: every stage state equals U^n, keep it bit for bit */
      A.out[v * nc + c] = A.Us[v * nc + c];
    } else {
      const double us = A.Us[v * nc + c];
      const double t1 = us + dt * r;
      A.out[v * nc + c] = (A.mode == 1) ? t1 : A.cA * A.U0[v * nc + c] + A.cB * t1;
    }
  }
}

struct StageArgs {
  CellUpdate cu;       /* faces of every axis, states, dt, 1/dx_a, stage coefficients */
  int n[3];
  long long ncell;
};

/* Flux difference -sum_a (F_{a,i+1/2} - F_{a,i-1/2})/dx_a (Eq. approximateEq) fused with
   the SSP-RK3 stage combine (cell_update); 1/dx_a is formed once on the host (an FP64 division per cell and axis
   would occupy the FP64 pipe longer than the kernel's memory traffic takes). */
template <int NV>
__global__ void stage_kernel(const StageArgs A) {
  constexpr int DIM = NV - 2;
  const long long nc = A.ncell;
  const double dt = (A.cu.mode != 0) ? *A.cu.dt : 0.0;
  /* one thread per cell: x from the block's column, y and z from the grid (strided when an
     axis exceeds the grid's 65535 limit) */
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= A.n[0]) return;
  for (int z = blockIdx.z; z < A.n[2]; z += gridDim.z) {
    for (int y = blockIdx.y; y < A.n[1]; y += gridDim.y) {
      const long long yz = y + (long long)A.n[1] * z;
      const long long c = x + (long long)A.n[0] * yz;
      long long fl[3] = {0, 0, 0}, fs[3] = {0, 0, 0};
      const long long fx = x + (long long)(A.n[0] + 1) * yz;
      if (DIM > 1) {
        fl[1] = x + (long long)A.n[0] * (y + (long long)(A.n[1] + 1) * z);
        fs[1] = A.n[0];
      }
      if (DIM > 2) {
        fl[2] = c;
        fs[2] = (long long)A.n[0] * A.n[1];
      }
      double dfx[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double* F = A.cu.F[0] + v * A.cu.nface[0];
        dfx[v] = F[fx + 1] - F[fx];
      }
      cell_update<NV>(A.cu, nc, c, dfx, fl, fs, dt);
    }
  }
}

static cudaError_t launch_stage_kernel(int nv, const StageArgs& a, cudaStream_t st) {
  const dim3 grid((unsigned)((a.n[0] + 255) / 256), (unsigned)(a.n[1] < 65535 ? a.n[1] : 65535),
                  (unsigned)(a.n[2] < 65535 ? a.n[2] : 65535));
  if (nv == 3) stage_kernel<3><<<grid, 256, 0, st>>>(a);
  else if (nv == 4) stage_kernel<4><<<grid, 256, 0, st>>>(a);
  else stage_kernel<5><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

/* max_i sum_a (|u_a| + c)/dx_a, reduced with atomicMax on the (positive) bit pattern. */
template <int NV>
__global__ void signal_speed_kernel(const double* __restrict__ U, long long nc, double gamma, double rdx0,
                                    double rdx1, double rdx2, unsigned long long* smax, int* status) {
  constexpr int DIM = NV - 2;
  const double rdx[3] = {rdx0, rdx1, rdx2};
  double m = 0.0;
  int st = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x) {
    const double rho = U[c];
    const double rinv = rcp_nr(rho);
    double vel[DIM], ke = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      vel[d] = U[(1 + d) * nc + c] * rinv;
      ke += U[(1 + d) * nc + c] * vel[d];
    }
    const double p = (gamma - 1.0) * (U[(NV - 1) * nc + c] - 0.5 * ke);
    if (!(rho > 0.0)) st |= ST_RHO;
    if (!(p > 0.0)) st |= ST_P;
    const double cs = sqrt(gamma * p * rinv);
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) s += (fabs(vel[d]) + cs) * rdx[d];
    m = (s > m) ? s : m;
  }
  /* warp then block reduction */
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  __shared__ double red[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = m;
  __syncthreads();
  if (w == 0) {
    m = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_xor_sync(0xffffffffu, m, o);
      m = t > m ? t : m;
    }
    if (l == 0 && m == m) atomicMax(smax, (unsigned long long)__double_as_longlong(m));
  }
  if (st) atomicOr(status, st);
}

/* dt = min(cfl / smax, t_end - t) (t_end = inf: no clip); resets smax for the next use. */
__global__ void finalize_dt_kernel(unsigned long long* smax, double cfl, double* dt_out, const double* t,
                                   double t_end) {
  const double s = __longlong_as_double((long long)*smax);
  double dt = cfl / s;
  if (t) {
    const double rem = t_end - *t;
    dt = rem < dt ? rem : dt;
    if (!(rem > 0.0)) dt = 0.0;
  }
  *dt_out = dt;
  *smax = 0ull;
}

__global__ void advance_time_kernel(double* t, const double* dt) { *t = *t + *dt; }

/* Compare the Newton-Raphson reciprocal / rsqrt with CUDA's correctly rounded 1.0/x, sqrt. */
/* per-cell primitives for the face sweeps of one stage: P = [velocity (NV-2), p, H, c, sqrt rho] */
template <int NV>
__global__ void prim_kernel(const double* __restrict__ U, long long ncell, double gamma, double* __restrict__ P,
                            int* status) {
  int st = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell; i += (long long)gridDim.x * blockDim.x) {
    double u[NV], vel[NV - 2], pr, Hh, c, sr;
#pragma unroll
    for (int q = 0; q < NV; ++q) u[q] = U[q * ncell + i];
    point_prims<NV>(u, gamma, vel, pr, Hh, c, sr, st);
#pragma unroll
    for (int d = 0; d < NV - 2; ++d) P[d * ncell + i] = vel[d];
    P[(NV - 2) * ncell + i] = pr;
    P[(NV - 1) * ncell + i] = Hh;
    P[NV * ncell + i] = c;
    P[(NV + 1) * ncell + i] = sr;
  }
  if (st) atomicOr(status, st);
}

/* Positivity-preserving flux limiter of one forward-Euler stage of length dt (Section 4.4),
   in place on the face fluxes of one axis, one thread per face; the per-face arithmetic is
   in tenom_positivity.cuh.  The cell outside a transmissive boundary is the boundary's copy
   of the edge cell, checked like an interior one. */
struct PosArgs {
  const double* U;
  double* F;           /* face fluxes of the axis, [NV][nface] */
  const double* dt;    /* device dt of the stage */
  int n[3];
  int bc[3];
  int axis;
  double mu_per_dt;    /* 2 dim / dx_a */
  double gamma;
};

/* The limiter proper at one face (cells c0 | c1, face lin), rarely reached; it re-reads its
   inputs (cached) rather than keeping the common path's values live. */
template <int NV, int AXIS>
__device__ __forceinline__ void limit_face(const PosArgs& A, long long c0, long long c1, long long lin, long long ncell,
                                           long long nface, double mu) {
  double Us[2][NV], F[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    Us[0][v] = A.U[v * ncell + c0];
    Us[1][v] = A.U[v * ncell + c1];
    F[v] = A.F[v * nface + lin];
  }
  if (limit_core<NV, AXIS>(Us, F, mu, A.gamma)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) A.F[v * nface + lin] = F[v];
  }
}

template <int NV, int AXIS>
__global__ void positivity_kernel(const PosArgs A) {
  const double dt = *A.dt;
  if (!(dt > 0.0)) return;  /* a step past t_end: nothing moves */
  const int fn0 = A.n[0] + (AXIS == 0), fn1 = A.n[1] + (AXIS == 1), fn2 = A.n[2] + (AXIS == 2);
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= fn0) return;
  const long long ncell = (long long)A.n[0] * A.n[1] * A.n[2];
  const long long nface = (long long)fn0 * fn1 * fn2;
  const double mu = A.mu_per_dt * dt;
  const double gm1 = A.gamma - 1.0;
  const float muf = f32_rz(mu), gm1f = f32_rz(gm1);
  const int na = A.n[AXIS];
  const bool periodic = A.bc[AXIS] == TENOM_BC_PERIODIC;
  const long long cstride = (AXIS == 0) ? 1 : (AXIS == 1 ? (long long)A.n[0] : (long long)A.n[0] * A.n[1]);
  for (int z = blockIdx.z; z < fn2; z += gridDim.z) {
    for (int y = blockIdx.y; y < fn1; y += gridDim.y) {
      const long long lin = x + (long long)fn0 * (y + (long long)fn1 * z);
      const int f = (AXIS == 0) ? x : (AXIS == 1 ? y : z);
      int jl = f - 1, jr = f;
      if (periodic) {
        if (jl < 0) jl += na;
        if (jr >= na) jr -= na;
      } else {
        if (jl < 0) jl = 0;
        if (jr > na - 1) jr = na - 1;
      }
      /* cell index of (x, y, z) with the AXIS coordinate set to 0 */
      const long long base = (AXIS == 0 ? 0 : x) + (long long)A.n[0] * ((AXIS == 1 ? 0 : y) +
                                                                       (long long)A.n[1] * (AXIS == 2 ? 0 : z));
      const long long c0 = base + jl * cstride, c1 = base + jr * cstride;
      /* early exit: when both one-sided states made with F^H have density and pressure
         (tested as rho p against 2e-13 rho, division-free) at least 2e-13, twice the largest
         floor, neither factor can fall below 1 and the face is left as it is.  First proven
         in FP32 (screen_fp32), else tested in FP64. */
      double FH[NV], Ua[NV], Ub[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        FH[v] = A.F[v * nface + lin];
        Ua[v] = A.U[v * ncell + c0];
        Ub[v] = A.U[v * ncell + c1];
      }
      if (screen_fp32<NV>(Ua, FH, -muf, gm1f) && screen_fp32<NV>(Ub, FH, muf, gm1f)) continue;
      if (!exit_fp64<NV>(Ua, Ub, FH, mu, gm1)) limit_face<NV, AXIS>(A, c0, c1, lin, ncell, nface, mu);
    }
  }
}

static cudaError_t launch_positivity_kernel(int nv, const PosArgs& p, cudaStream_t st) {
  int fn[3] = {p.n[0], p.n[1], p.n[2]};
  fn[p.axis] += 1;
  const dim3 grid((unsigned)((fn[0] + 127) / 128), (unsigned)(fn[1] < 65535 ? fn[1] : 65535),
                  (unsigned)(fn[2] < 65535 ? fn[2] : 65535));
  if (nv == 3) positivity_kernel<3, 0><<<grid, 128, 0, st>>>(p);
  else if (nv == 4) {
    if (p.axis == 0) positivity_kernel<4, 0><<<grid, 128, 0, st>>>(p);
    else positivity_kernel<4, 1><<<grid, 128, 0, st>>>(p);
  } else {
    if (p.axis == 0) positivity_kernel<5, 0><<<grid, 128, 0, st>>>(p);
    else if (p.axis == 1) positivity_kernel<5, 1><<<grid, 128, 0, st>>>(p);
    else positivity_kernel<5, 2><<<grid, 128, 0, st>>>(p);
  }
  return cudaGetLastError();
}

__global__ void fastmath_check_kernel(const double* x, double* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    out[6 * i + 0] = rcp_nr(v);
    out[6 * i + 1] = 1.0 / v;
    const double r = rsqrt_nr(v);
    out[6 * i + 2] = v * r;
    out[6 * i + 3] = sqrt(v);
    out[6 * i + 4] = rcp_nr1(v);
    out[6 * i + 5] = (double)f32_rz((i & 1) ? -v : v);
  }
}

/* out = c0 x0 + c1 x1 + c2 x2 + c3 dt x3 (null operands skipped; dt read on the device) */
__global__ void lincomb_kernel(long long n, double* out, double c0, const double* x0, double c1, const double* x1,
                               double c2, const double* x2, double c3, const double* dtp, const double* x3) {
  const double dt = dtp ? *dtp : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double r = c0 * x0[i];
    if (x1) r += c1 * x1[i];
    if (x2) r += c2 * x2[i];
    if (x3) r += (c3 * dt) * x3[i];
    out[i] = r;
  }
}

/* FP64 pipe probe: 8 independent FMA chains per thread. */
__global__ void dfma_probe_kernel(int iters, double a, double b, double* sink) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 12345.678) sink[0] = s;  /* keeps the chains live */
}

}  // namespace tenom

using namespace tenom;

/* ---------------------------------------------------------------- context */

struct tenom_ctx {
  tenom_grid g;
  tenom_scheme s;
  cudaStream_t st;
  int nv;
  long long ncell;
  long long nface[3];
  double* W1;          /* stage buffer */
  double* face[3];     /* face buffers */
  double* P;           /* per-cell primitives of the stage being evaluated ([nvar + 2][ncell]) */
  double* dt;          /* device dt */
  double* tbuf;        /* device scratch time */
  double* Uhost;       /* device state for tenom_advance_host (allocated on first use) */
  double* adj;         /* adjoint workspace: A1, A2, A3, Z, then an internal tape (U^n copy, U1, U2) */
  uint8_t* adj_flags;  /* internal tape flags (3 stages) */
  unsigned long long* smax;
  int* status;
  std::string err;
  bool timing;
  std::vector<cudaEvent_t> ev;  /* pairs around face launches */
  size_t ev_used;
  double face_ms;
  long long face_launches;
};

static tenom_status fail(tenom_ctx* c, tenom_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

static tenom_status cuda_fail(tenom_ctx* c, cudaError_t e, const char* where) {
  return fail(c, TENOM_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static const double kDopt6[4] = {9.0 / 20.0, 3.0 / 10.0, 1.0 / 20.0, 1.0 / 5.0};
static const double kDopt8[6] = {3.0 / 7.0, 9.0 / 35.0, 2.0 / 35.0, 6.0 / 35.0, 1.0 / 70.0, 1.0 / 14.0};

static SchemeDev scheme_dev(const tenom_scheme& s) {
  SchemeDev d;
  memset(&d, 0, sizeof(d));
  d.ct_mode = s.ct_mode;
  d.mp_curv = s.mp_curv;
  d.weights = s.weights;
  d.ct_const = s.ct_const;
  d.mp_alpha = s.mp_alpha;
  d.mp_beta_third = s.mp_beta / 3.0;
  for (int k = 0; k < 6; ++k) d.d[k] = s.d[k];
  d.exact_decisions = (s.decisions == TENOM_DECIDE_FP64) ? 1 : 0;
  d.ct_const_f = (float)s.ct_const;
  d.default_d = 1;
  for (int k = 0; k < s.K - 2; ++k)
    if (s.d[k] != ((s.K == 6) ? kDopt6[k] : kDopt8[k])) d.default_d = 0;
  return d;
}


extern "C" {

tenom_status tenom_scheme_default(tenom_scheme* s, int K) {
  if (!s || (K != 6 && K != 8)) return TENOM_E_INVALID;
  memset(s, 0, sizeof(*s));
  s->K = K;
  s->limiter = TENOM_LIM_MP;
  s->ct_mode = (K == 6) ? TENOM_CT_CONST : TENOM_CT_ADAPTIVE;
  s->ct_const = 1e-5;
  s->mp_alpha = 1.25;
  s->mp_beta = 4.0;
  s->mp_curv = TENOM_CURV_M4;
  s->weights = TENOM_W_TENOM;
  for (int k = 0; k < K - 2; ++k) s->d[k] = (K == 6) ? kDopt6[k] : kDopt8[k];
  return TENOM_OK;
}

static tenom_status validate(const tenom_grid* g, const tenom_scheme* s, std::string* msg) {
  if (!g || !s) { *msg = "null grid or scheme"; return TENOM_E_INVALID; }
  if (g->dim < 1 || g->dim > 3) { *msg = "dim must be 1, 2 or 3"; return TENOM_E_INVALID; }
  for (int a = 0; a < 3; ++a) {
    if (a < g->dim) {
      if (g->n[a] < 1 || g->n[a] > (1 << 24)) { *msg = "cell count out of range"; return TENOM_E_INVALID; }
      if (!(g->dx[a] > 0.0) || !std::isfinite(g->dx[a])) { *msg = "dx must be positive"; return TENOM_E_INVALID; }
      if (g->bc[a] != TENOM_BC_PERIODIC && g->bc[a] != TENOM_BC_TRANSMISSIVE) { *msg = "bad bc"; return TENOM_E_INVALID; }
    } else if (g->n[a] != 1) {
      *msg = "unused axes must have n = 1";
      return TENOM_E_INVALID;
    }
  }
  if (!(g->gamma > 1.0)) { *msg = "gamma must exceed 1"; return TENOM_E_INVALID; }
  long long nc = (long long)g->n[0] * g->n[1] * g->n[2];
  if (nc > (1ll << 31)) { *msg = "grid too large"; return TENOM_E_INVALID; }
  if (g->dim > 1 && (long long)g->n[1] * g->n[2] > 2147483647ll) { *msg = "too many rows"; return TENOM_E_INVALID; }
  if (s->K != 6 && s->K != 8) { *msg = "K must be 6 or 8"; return TENOM_E_INVALID; }
  if (s->limiter != TENOM_LIM_MP && s->limiter != TENOM_LIM_TVD5 && s->limiter != TENOM_LIM_VA) {
    *msg = "bad limiter";
    return TENOM_E_INVALID;
  }
  if (s->ct_mode != TENOM_CT_CONST && s->ct_mode != TENOM_CT_ADAPTIVE) { *msg = "bad ct_mode"; return TENOM_E_INVALID; }
  if (s->mp_curv != TENOM_CURV_M4 && s->mp_curv != TENOM_CURV_MM) { *msg = "bad mp_curv"; return TENOM_E_INVALID; }
  if (s->weights != TENOM_W_TENOM && s->weights != TENOM_W_TENO) { *msg = "bad weights"; return TENOM_E_INVALID; }
  if (s->positivity != TENOM_PP_OFF && s->positivity != TENOM_PP_ON) { *msg = "bad positivity flag"; return TENOM_E_INVALID; }
  if (s->decisions != TENOM_DECIDE_FILTERED && s->decisions != TENOM_DECIDE_FP64) {
    *msg = "bad decisions mode";
    return TENOM_E_INVALID;
  }
  for (int a = 0; a < g->dim; ++a)
    if (g->n[a] < s->K / 2 && g->bc[a] == TENOM_BC_PERIODIC) {
      *msg = "periodic axis shorter than the half stencil";
      return TENOM_E_INVALID;
    }
  return TENOM_OK;
}

tenom_status tenom_create(tenom_ctx** out, const tenom_grid* grid, const tenom_scheme* scheme, void* stream) {
  if (!out) return TENOM_E_INVALID;
  *out = nullptr;
  std::string msg;
  tenom_status v = validate(grid, scheme, &msg);
  if (v != TENOM_OK) {
    fprintf(stderr, "tenom_create: %s\n", msg.c_str());
    return v;
  }
  tenom_ctx* c = new tenom_ctx();
  c->g = *grid;
  c->s = *scheme;
  bool anyd = false;
  for (int k = 0; k < 6; ++k) anyd |= (c->s.d[k] != 0.0);
  if (!anyd)
    for (int k = 0; k < c->s.K - 2; ++k) c->s.d[k] = (c->s.K == 6) ? kDopt6[k] : kDopt8[k];
  c->st = (cudaStream_t)stream;
  c->nv = grid->dim + 2;
  c->ncell = (long long)grid->n[0] * grid->n[1] * grid->n[2];
  for (int a = 0; a < 3; ++a) {
    c->nface[a] = 0;
    c->face[a] = nullptr;
    if (a < grid->dim) c->nface[a] = c->ncell / grid->n[a] * (grid->n[a] + 1);
  }
  c->Uhost = nullptr;
  c->adj = nullptr;
  c->adj_flags = nullptr;
  c->timing = false;
  c->ev_used = 0;
  c->face_ms = 0;
  c->face_launches = 0;
  cudaError_t e = cudaMalloc(&c->W1, sizeof(double) * c->nv * c->ncell);
  for (int a = 0; a < grid->dim && e == cudaSuccess; ++a) e = cudaMalloc(&c->face[a], sizeof(double) * c->nv * c->nface[a]);
  if (e == cudaSuccess) e = cudaMalloc(&c->P, sizeof(double) * (c->nv + 2) * c->ncell);
  if (e == cudaSuccess) e = cudaMalloc(&c->dt, sizeof(double) * 2);
  if (e == cudaSuccess) e = cudaMalloc(&c->smax, sizeof(unsigned long long) + sizeof(int) * 2);
  if (e == cudaSuccess) {
    c->tbuf = c->dt + 1;
    c->status = (int*)(c->smax + 1);
    e = cudaMemsetAsync(c->smax, 0, sizeof(unsigned long long) + sizeof(int) * 2, c->st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->dt, 0, sizeof(double) * 2, c->st);
  if (e != cudaSuccess) {
    fprintf(stderr, "tenom_create: %s\n", cudaGetErrorString(e));
    tenom_destroy(c);
    return TENOM_E_CUDA;
  }
  *out = c;
  return TENOM_OK;
}

tenom_status tenom_destroy(tenom_ctx* c) {
  if (!c) return TENOM_OK;
  cudaStreamSynchronize(c->st);
  cudaFree(c->W1);
  for (int a = 0; a < 3; ++a) cudaFree(c->face[a]);
  cudaFree(c->P);
  cudaFree(c->dt);
  cudaFree(c->smax);
  cudaFree(c->Uhost);
  cudaFree(c->adj);
  cudaFree(c->adj_flags);
  for (cudaEvent_t ev : c->ev) cudaEventDestroy(ev);
  delete c;
  return TENOM_OK;
}

const char* tenom_last_error(const tenom_ctx* c) { return c ? c->err.c_str() : ""; }

static bool aligned8(const void* p) { return p && ((uintptr_t)p & 7) == 0; }

static unsigned ew_blocks(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

tenom_status tenom_init_state(tenom_ctx* c, const double* prim, double* U) {
  if (!c) return TENOM_E_INVALID;
  if (!aligned8(prim) || !aligned8(U) || prim == U) return fail(c, TENOM_E_INVALID, "init_state: bad pointers");
  unsigned nb = ew_blocks(c->ncell);
  if (c->nv == 3) init_state_kernel<3><<<nb, 256, 0, c->st>>>(prim, U, c->ncell, c->g.gamma);
  else if (c->nv == 4) init_state_kernel<4><<<nb, 256, 0, c->st>>>(prim, U, c->ncell, c->g.gamma);
  else init_state_kernel<5><<<nb, 256, 0, c->st>>>(prim, U, c->ncell, c->g.gamma);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, "init_state");
}

static FaceArgs face_args(tenom_ctx* c, const double* U, int axis, double* F, uint8_t* flags) {
  FaceArgs a;
  memset(&a, 0, sizeof(a));
  a.U = U;
  a.Fhat = F;
  a.flags = flags;
  a.status = c->status;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = c->g.n[d];
    a.bc[d] = c->g.bc[d];
  }
  a.ncell = c->ncell;
  a.nface = c->nface[axis];
  a.gamma = c->g.gamma;
  a.sch = scheme_dev(c->s);
  return a;
}

/* one face sweep of axis `axis` at U (P: its cell primitives) */
static cudaError_t launch_faces(tenom_ctx* c, const double* U, int axis, double* F, uint8_t* flags,
                                double* lin = nullptr, const double* P = nullptr) {
  FaceArgs a = face_args(c, U, axis, F, flags);
  a.lin = lin;
  a.P = P;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing) {
    while (c->ev.size() < c->ev_used + 2) {
      cudaEvent_t ev;
      cudaError_t er = cudaEventCreate(&ev);
      if (er != cudaSuccess) return er;
      c->ev.push_back(ev);
    }
    e0 = c->ev[c->ev_used];
    e1 = c->ev[c->ev_used + 1];
    c->ev_used += 2;
    cudaEventRecord(e0, c->st);
  }
  cudaError_t e;
  if (lin) {
    if (c->nv == 3) e = launch_face_rec_nv3(a, axis, c->s.K, c->s.limiter, c->st);
    else if (c->nv == 4) e = launch_face_rec_nv4(a, axis, c->s.K, c->s.limiter, c->st);
    else e = launch_face_rec_nv5(a, axis, c->s.K, c->s.limiter, c->st);
  } else {
    if (c->nv == 3) e = launch_face_nv3(a, axis, c->s.K, c->s.limiter, c->st);
    else if (c->nv == 4) e = launch_face_nv4(a, axis, c->s.K, c->s.limiter, c->st);
    else e = launch_face_nv5(a, axis, c->s.K, c->s.limiter, c->st);
  }
  if (c->timing) cudaEventRecord(e1, c->st);
  return e;
}

static CellUpdate cell_update_args(tenom_ctx* c, const double* U0, const double* Us, double* out, int mode, double cA,
                                   double cB) {
  CellUpdate u;
  memset(&u, 0, sizeof(u));
  for (int d = 0; d < 3; ++d) {
    u.F[d] = c->face[d];
    u.rdx[d] = 1.0 / c->g.dx[d];
    u.nface[d] = c->nface[d];
  }
  u.U0 = U0;
  u.Us = Us;
  u.out = out;
  u.dt = c->dt;
  u.cA = cA;
  u.cB = cB;
  u.mode = mode;
  return u;
}

static cudaError_t launch_stage(tenom_ctx* c, const double* U0, const double* Us, double* out, int mode, double cA,
                                double cB) {
  StageArgs a;
  memset(&a, 0, sizeof(a));
  a.cu = cell_update_args(c, U0, Us, out, mode, cA, cB);
  for (int d = 0; d < 3; ++d) a.n[d] = c->g.n[d];
  a.ncell = c->ncell;
  return launch_stage_kernel(c->nv, a, c->st);
}

/* the cell primitives of U into c->P (read by the face sweeps of this stage) */
static cudaError_t launch_prims(tenom_ctx* c, const double* U) {
  const unsigned nb = ew_blocks(c->ncell);
  if (c->nv == 3) prim_kernel<3><<<nb, 256, 0, c->st>>>(U, c->ncell, c->g.gamma, c->P, c->status);
  else if (c->nv == 4) prim_kernel<4><<<nb, 256, 0, c->st>>>(U, c->ncell, c->g.gamma, c->P, c->status);
  else prim_kernel<5><<<nb, 256, 0, c->st>>>(U, c->ncell, c->g.gamma, c->P, c->status);
  return cudaGetLastError();
}

/* face fluxes of every axis at U: the cell primitives once, then one sweep per axis */
static cudaError_t eval_faces(tenom_ctx* c, const double* U) {
  cudaError_t e = launch_prims(c, U);
  for (int a = 0; a < c->g.dim && e == cudaSuccess; ++a) e = launch_faces(c, U, a, c->face[a], nullptr, nullptr, c->P);
  return e;
}

tenom_status tenom_rhs(tenom_ctx* c, const double* U, double* dUdt) {
  if (!c) return TENOM_E_INVALID;
  if (!aligned8(U) || !aligned8(dUdt) || U == dUdt) return fail(c, TENOM_E_INVALID, "rhs: bad pointers");
  cudaError_t e = eval_faces(c, U);
  if (e == cudaSuccess) e = launch_stage(c, nullptr, U, dUdt, 0, 0.0, 0.0);
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, "rhs");
}

static cudaError_t launch_signal(tenom_ctx* c, const double* U) {
  unsigned nb = ew_blocks(c->ncell);
  const double* dx = c->g.dx;
  const double r0 = 1.0 / dx[0], r1 = 1.0 / dx[1], r2 = 1.0 / dx[2];
  if (c->nv == 3) signal_speed_kernel<3><<<nb, 256, 0, c->st>>>(U, c->ncell, c->g.gamma, r0, r1, r2, c->smax, c->status);
  else if (c->nv == 4) signal_speed_kernel<4><<<nb, 256, 0, c->st>>>(U, c->ncell, c->g.gamma, r0, r1, r2, c->smax, c->status);
  else signal_speed_kernel<5><<<nb, 256, 0, c->st>>>(U, c->ncell, c->g.gamma, r0, r1, r2, c->smax, c->status);
  return cudaGetLastError();
}

tenom_status tenom_max_dt(tenom_ctx* c, const double* U, double cfl, double* dt_dev) {
  if (!c) return TENOM_E_INVALID;
  if (!aligned8(U) || !aligned8(dt_dev) || !(cfl > 0.0)) return fail(c, TENOM_E_INVALID, "max_dt: bad arguments");
  cudaError_t e = launch_signal(c, U);
  if (e == cudaSuccess) {
    finalize_dt_kernel<<<1, 1, 0, c->st>>>(c->smax, cfl, dt_dev, nullptr, 0.0);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, "max_dt");
}

/* the positivity limiter on the face fluxes F of axis a, computed from the state Us, for a
   forward-Euler stage of length *dt */
static cudaError_t launch_positivity_axis(tenom_ctx* c, const double* Us, int a, const double* dt, double* F) {
  PosArgs p;
  memset(&p, 0, sizeof(p));
  p.U = Us;
  p.F = F;
  p.dt = dt;
  for (int d = 0; d < 3; ++d) {
    p.n[d] = c->g.n[d];
    p.bc[d] = c->g.bc[d];
  }
  p.axis = a;
  p.mu_per_dt = 2.0 * c->g.dim / c->g.dx[a];
  p.gamma = c->g.gamma;
  return launch_positivity_kernel(c->nv, p, c->st);
}

/* the positivity limiter on every axis's face fluxes of the stage at Us (length c->dt) */
static cudaError_t launch_positivity(tenom_ctx* c, const double* Us) {
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < c->g.dim && e == cudaSuccess; ++a) e = launch_positivity_axis(c, Us, a, c->dt, c->face[a]);
  return e;
}

/* face fluxes of one SSP-RK3 stage at Us: the high-order fluxes, limited when the scheme
   asks for positivity */
static cudaError_t stage_faces(tenom_ctx* c, const double* Us) {
  cudaError_t e = eval_faces(c, Us);
  if (e == cudaSuccess && c->s.positivity == TENOM_PP_ON) e = launch_positivity(c, Us);
  return e;
}

/* three stages; dt already in c->dt */
static cudaError_t rk3_core(tenom_ctx* c, double* U) {
  cudaError_t e = stage_faces(c, U);
  if (e == cudaSuccess) e = launch_stage(c, nullptr, U, c->W1, 1, 0.0, 1.0);
  if (e == cudaSuccess) e = stage_faces(c, c->W1);
  if (e == cudaSuccess) e = launch_stage(c, U, c->W1, c->W1, 2, 0.75, 0.25);
  if (e == cudaSuccess) e = stage_faces(c, c->W1);
  if (e == cudaSuccess) e = launch_stage(c, U, c->W1, U, 2, 1.0 / 3.0, 2.0 / 3.0);
  return e;
}

tenom_status tenom_rk3_step(tenom_ctx* c, double* U, const double* dt_dev) {
  if (!c) return TENOM_E_INVALID;
  if (!aligned8(U) || !aligned8(dt_dev)) return fail(c, TENOM_E_INVALID, "rk3_step: bad pointers");
  cudaError_t e = cudaSuccess;
  if (dt_dev != c->dt) e = cudaMemcpyAsync(c->dt, dt_dev, sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess) e = rk3_core(c, U);
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, "rk3_step");
}

tenom_status tenom_advance(tenom_ctx* c, double* U, double* t_dev, double t_end, double cfl, int nsteps) {
  if (!c) return TENOM_E_INVALID;
  if (!aligned8(U) || !aligned8(t_dev) || !(cfl > 0.0) || nsteps < 0 || !(t_end == t_end))
    return fail(c, TENOM_E_INVALID, "advance: bad arguments");
  for (int k = 0; k < nsteps; ++k) {
    cudaError_t e = launch_signal(c, U);
    if (e == cudaSuccess) {
      finalize_dt_kernel<<<1, 1, 0, c->st>>>(c->smax, cfl, c->dt, t_dev, t_end);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = rk3_core(c, U);
    if (e == cudaSuccess) {
      advance_time_kernel<<<1, 1, 0, c->st>>>(t_dev, c->dt);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "advance");
  }
  return TENOM_OK;
}

tenom_status tenom_advance_host(tenom_ctx* c, const double* U_in, double* U_out, double* t_host, double t_end,
                                double cfl, int nsteps) {
  if (!c) return TENOM_E_INVALID;
  if (!U_in || !U_out || !t_host) return fail(c, TENOM_E_INVALID, "advance_host: null pointer");
  size_t bytes = sizeof(double) * c->nv * c->ncell;
  cudaError_t e = cudaSuccess;
  if (!c->Uhost) e = cudaMalloc(&c->Uhost, bytes);
  double* Ud = c->Uhost;
  if (e == cudaSuccess) e = cudaMemcpyAsync(Ud, U_in, bytes, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->tbuf, t_host, sizeof(double), cudaMemcpyHostToDevice, c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "advance_host");
  tenom_status s = tenom_advance(c, Ud, c->tbuf, t_end, cfl, nsteps);
  if (s == TENOM_OK) {
    e = cudaMemcpyAsync(U_out, Ud, bytes, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t_host, c->tbuf, sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "advance_host");
  }
  return s;
}

tenom_status tenom_positivity_limit(tenom_ctx* c, const double* U, int axis, const double* dt_dev, double* Fhat) {
  if (!c) return TENOM_E_INVALID;
  if (axis < 0 || axis >= c->g.dim) return fail(c, TENOM_E_INVALID, "positivity_limit: bad axis");
  if (!aligned8(U) || !aligned8(dt_dev) || !aligned8(Fhat)) return fail(c, TENOM_E_INVALID, "positivity_limit: bad pointers");
  cudaError_t e = launch_positivity_axis(c, U, axis, dt_dev, Fhat);
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, "positivity_limit");
}

tenom_status tenom_face_dump(tenom_ctx* c, const double* U, int axis, double* Fhat, uint8_t* flags) {
  if (!c) return TENOM_E_INVALID;
  if (axis < 0 || axis >= c->g.dim) return fail(c, TENOM_E_INVALID, "face_dump: bad axis");
  if (!aligned8(U) || !aligned8(Fhat)) return fail(c, TENOM_E_INVALID, "face_dump: bad pointers");
  bool t = c->timing;
  c->timing = false;
  cudaError_t e = launch_faces(c, U, axis, Fhat, flags);
  c->timing = t;
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, "face_dump");
}

tenom_status tenom_decision_stats(tenom_ctx* c, const double* U, int axis, unsigned long long* counters_dev) {
  static_assert(TENOM_NSTATS == SC_COUNT, "counter layout of the header and the kernels");
  if (!c) return TENOM_E_INVALID;
  if (axis < 0 || axis >= c->g.dim) return fail(c, TENOM_E_INVALID, "decision_stats: bad axis");
  if (!aligned8(U) || !aligned8(counters_dev)) return fail(c, TENOM_E_INVALID, "decision_stats: bad pointers");
  cudaError_t e = launch_prims(c, U);
  if (e == cudaSuccess) {
    FaceArgs a = face_args(c, U, axis, nullptr, nullptr);
    a.P = c->P;
    a.stats = counters_dev;
    if (c->nv == 3) e = launch_stats_nv3(a, axis, c->s.K, c->s.limiter, c->st);
    else if (c->nv == 4) e = launch_stats_nv4(a, axis, c->s.K, c->s.limiter, c->st);
    else e = launch_stats_nv5(a, axis, c->s.K, c->s.limiter, c->st);
  }
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, "decision_stats");
}

tenom_status tenom_status_word(tenom_ctx* c, int* status_host, int reset) {
  if (!c || !status_host) return TENOM_E_INVALID;
  cudaError_t e = cudaMemcpyAsync(status_host, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "status_word");
  return *status_host ? TENOM_E_NONPHYSICAL : TENOM_OK;
}

tenom_status tenom_kernel_timing(tenom_ctx* c, int enable, double* face_ms_per_launch, long long* launches) {
  if (!c) return TENOM_E_INVALID;
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel_timing");
  double tot = 0.0;
  long long n = 0;
  for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]) == cudaSuccess) {
      tot += ms;
      ++n;
    }
  }
  if (face_ms_per_launch) *face_ms_per_launch = n ? tot / n : 0.0;
  if (launches) *launches = n;
  c->ev_used = 0;
  c->timing = enable != 0;
  return TENOM_OK;
}

/* ---------------------------------------------------------------- adjoint */

size_t tenom_flags_bytes(const tenom_ctx* c) {
  if (!c) return 0;
  size_t b = 0;
  for (int a = 0; a < c->g.dim; ++a) b += (size_t)c->nface[a] * c->nv * 2;
  return b;
}

static size_t flags_offset(const tenom_ctx* c, int axis) {
  size_t b = 0;
  for (int a = 0; a < axis; ++a) b += (size_t)c->nface[a] * c->nv * 2;
  return b;
}

/* The frozen-branch adjoint covers the limiters whose filtered candidate is a selection
   among linear forms (MP, TVD5); the Van Albada flux is a smooth nonlinear function of the
   stencil and has no frozen linear form here, nor has the positivity limiter's blend
   factor (a ratio of the states' densities and pressures). */
static bool adjoint_unsupported(tenom_ctx* c, const char* what) {
  if (c->s.limiter == TENOM_LIM_VA) {
    fail(c, TENOM_E_UNSUPPORTED, std::string(what) + ": no adjoint for the Van Albada limiter");
    return true;
  }
  if (c->s.positivity == TENOM_PP_ON) {
    fail(c, TENOM_E_UNSUPPORTED, std::string(what) + ": no adjoint for the positivity limiter");
    return true;
  }
  return false;
}

/* doubles of the linearisation one stage records for one face: NV x (2K + 2) */
static size_t lin_per_face(const tenom_ctx* c) { return (size_t)c->nv * (2 * c->s.K + 2); }

size_t tenom_lin_tape_bytes(const tenom_ctx* c) {
  if (!c) return 0;
  size_t b = 0;
  for (int a = 0; a < c->g.dim; ++a) b += (size_t)c->nface[a] * lin_per_face(c) * sizeof(double);
  return b;
}

/* offset, in doubles, of axis `axis` inside one stage's linearisation */
static size_t lin_offset(const tenom_ctx* c, int axis) {
  size_t b = 0;
  for (int a = 0; a < axis; ++a) b += (size_t)c->nface[a] * lin_per_face(c);
  return b;
}

static cudaError_t adj_sweeps(tenom_ctx* c, const double* U, const uint8_t* flags_stage, const double* lin_stage,
                              const double* w, double* Z) {
  cudaError_t e = cudaMemsetAsync(Z, 0, sizeof(double) * c->nv * c->ncell, c->st);
  if (e == cudaSuccess) e = launch_prims(c, U);
  for (int a = 0; a < c->g.dim && e == cudaSuccess; ++a) {
    AdjArgs A;
    memset(&A, 0, sizeof(A));
    A.U = U;
    A.flags = flags_stage ? flags_stage + flags_offset(c, a) : nullptr;
    A.lin = lin_stage ? lin_stage + lin_offset(c, a) : nullptr;
    A.P = c->P;
    A.w = w;
    A.Z = Z;
    A.status = c->status;
    for (int d = 0; d < 3; ++d) {
      A.n[d] = c->g.n[d];
      A.bc[d] = c->g.bc[d];
    }
    A.ncell = c->ncell;
    A.nface = c->nface[a];
    A.dx = c->g.dx[a];
    A.gamma = c->g.gamma;
    A.sch = scheme_dev(c->s);
    if (c->nv == 3) e = launch_adj_nv3(A, a, c->s.K, c->s.limiter, c->st);
    else if (c->nv == 4) e = launch_adj_nv4(A, a, c->s.K, c->s.limiter, c->st);
    else e = launch_adj_nv5(A, a, c->s.K, c->s.limiter, c->st);
  }
  return e;
}

static cudaError_t ensure_adj(tenom_ctx* c) {
  if (c->adj) return cudaSuccess;
  cudaError_t e = cudaMalloc(&c->adj, sizeof(double) * c->nv * c->ncell * 7);
  if (e == cudaSuccess) e = cudaMalloc(&c->adj_flags, tenom_flags_bytes(c) * 3);
  return e;
}

static cudaError_t lincomb(tenom_ctx* c, double* out, double c0, const double* x0, double c1, const double* x1,
                           double c2, const double* x2, double c3, const double* dtp, const double* x3) {
  const long long n = c->nv * c->ncell;
  lincomb_kernel<<<ew_blocks(n), 256, 0, c->st>>>(n, out, c0, x0, c1, x1, c2, x2, c3, dtp, x3);
  return cudaGetLastError();
}

tenom_status tenom_rhs_vjp(tenom_ctx* c, const double* U, const double* w, double* Ubar) {
  if (!c) return TENOM_E_INVALID;
  if (adjoint_unsupported(c, "rhs_vjp")) return TENOM_E_UNSUPPORTED;
  if (!aligned8(U) || !aligned8(w) || !aligned8(Ubar) || Ubar == U || Ubar == w)
    return fail(c, TENOM_E_INVALID, "rhs_vjp: bad pointers");
  cudaError_t e = adj_sweeps(c, U, nullptr, nullptr, w, Ubar);
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, "rhs_vjp");
}

tenom_status tenom_rhs_record(tenom_ctx* c, const double* U, double* dUdt, double* lin) {
  if (!c) return TENOM_E_INVALID;
  if (adjoint_unsupported(c, "rhs_record")) return TENOM_E_UNSUPPORTED;
  if (!aligned8(U) || !aligned8(dUdt) || U == dUdt || !aligned8(lin))
    return fail(c, TENOM_E_INVALID, "rhs_record: bad pointers");
  cudaError_t e = launch_prims(c, U);
  for (int a = 0; a < c->g.dim && e == cudaSuccess; ++a)
    e = launch_faces(c, U, a, c->face[a], nullptr, lin + lin_offset(c, a), c->P);
  if (e == cudaSuccess) e = launch_stage(c, nullptr, U, dUdt, 0, 0.0, 0.0);
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, "rhs_record");
}

tenom_status tenom_rhs_vjp_lin(tenom_ctx* c, const double* U, const double* lin, const double* w, double* Ubar) {
  if (!c) return TENOM_E_INVALID;
  if (adjoint_unsupported(c, "rhs_vjp_lin")) return TENOM_E_UNSUPPORTED;
  if (!aligned8(U) || !aligned8(lin) || !aligned8(w) || !aligned8(Ubar) || Ubar == U || Ubar == w)
    return fail(c, TENOM_E_INVALID, "rhs_vjp_lin: bad pointers");
  cudaError_t e = adj_sweeps(c, U, nullptr, lin, w, Ubar);
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, "rhs_vjp_lin");
}

/* one SSP-RK3 step that keeps its stage states and its cutoff flags (fl) or linearisation (lin) */
static cudaError_t rk3_record(tenom_ctx* c, double* U, double* U1, double* U2, uint8_t* fl, double* lin) {
  const size_t fb = tenom_flags_bytes(c);
  const size_t lb = tenom_lin_tape_bytes(c) / sizeof(double);
  const double* src[3] = {U, U1, U2};
  cudaError_t e = cudaSuccess;
  for (int st = 0; st < 3 && e == cudaSuccess; ++st) {
    e = launch_prims(c, src[st]);
    for (int a = 0; a < c->g.dim && e == cudaSuccess; ++a)
      e = launch_faces(c, src[st], a, c->face[a], fl ? fl + st * fb + flags_offset(c, a) : nullptr,
                       lin ? lin + st * lb + lin_offset(c, a) : nullptr, c->P);
    if (e != cudaSuccess) break;
    if (st == 0) e = launch_stage(c, nullptr, U, U1, 1, 0.0, 1.0);
    else if (st == 1) e = launch_stage(c, U, U1, U2, 2, 0.75, 0.25);
    else e = launch_stage(c, U, U2, U, 2, 1.0 / 3.0, 2.0 / 3.0);
  }
  return e;
}

static tenom_status record_step(tenom_ctx* c, double* U, const double* dt_dev, double* tape_states, uint8_t* fl,
                                double* lin, const char* what) {
  if (adjoint_unsupported(c, what)) return TENOM_E_UNSUPPORTED;
  cudaError_t e = cudaSuccess;
  if (dt_dev != c->dt) e = cudaMemcpyAsync(c->dt, dt_dev, sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  const long long n = c->nv * c->ncell;
  if (e == cudaSuccess) e = rk3_record(c, U, tape_states, tape_states + n, fl, lin);
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, what);
}

tenom_status tenom_rk3_step_record(tenom_ctx* c, double* U, const double* dt_dev, double* tape_states,
                                   uint8_t* tape_flags) {
  if (!c) return TENOM_E_INVALID;
  if (!aligned8(U) || !aligned8(dt_dev) || !aligned8(tape_states) || !tape_flags)
    return fail(c, TENOM_E_INVALID, "rk3_step_record: bad pointers");
  return record_step(c, U, dt_dev, tape_states, tape_flags, nullptr, "rk3_step_record");
}

tenom_status tenom_rk3_step_record_lin(tenom_ctx* c, double* U, const double* dt_dev, double* tape_states,
                                       double* tape_lin) {
  if (!c) return TENOM_E_INVALID;
  if (!aligned8(U) || !aligned8(dt_dev) || !aligned8(tape_states) || !aligned8(tape_lin))
    return fail(c, TENOM_E_INVALID, "rk3_step_record_lin: bad pointers");
  return record_step(c, U, dt_dev, tape_states, nullptr, tape_lin, "rk3_step_record_lin");
}

/* reverse of one recorded step; per stage the sweeps read flags (fl) or the linearisation (lin) */
static tenom_status adjoint_step(tenom_ctx* c, const double* U_n, const double* tape_states, const uint8_t* fl,
                                 const double* lin, const double* dt_dev, const double* Ubar_np1, double* Ubar_n) {
  if (adjoint_unsupported(c, "rk3_step_adjoint")) return TENOM_E_UNSUPPORTED;
  cudaError_t e = ensure_adj(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "rk3_step_adjoint");
  const long long n = c->nv * c->ncell;
  const size_t fb = tenom_flags_bytes(c);
  const size_t lb = tenom_lin_tape_bytes(c) / sizeof(double);
  auto F = [&](int st) { return fl ? fl + st * fb : nullptr; };
  auto Lz = [&](int st) { return lin ? lin + st * lb : nullptr; };
  double *A1 = c->adj, *A2 = c->adj + n, *A3 = c->adj + 2 * n, *Z = c->adj + 3 * n;
  const double *U1 = tape_states, *U2 = tape_states + n;
  /* stage 3: U^{n+1} = 1/3 U^n + 2/3 (U2 + dt L(U2)) */
  e = lincomb(c, A1, 2.0 / 3.0, Ubar_np1, 0, nullptr, 0, nullptr, 0, nullptr, nullptr);
  if (e == cudaSuccess) e = adj_sweeps(c, U2, F(2), Lz(2), A1, Z);
  if (e == cudaSuccess) e = lincomb(c, A2, 1.0, A1, 0, nullptr, 0, nullptr, 1.0, dt_dev, Z);    /* Ubar2 */
  /* stage 2: U2 = 3/4 U^n + 1/4 (U1 + dt L(U1)) */
  if (e == cudaSuccess) e = lincomb(c, A3, 0.25, A2, 0, nullptr, 0, nullptr, 0, nullptr, nullptr);
  if (e == cudaSuccess) e = adj_sweeps(c, U1, F(1), Lz(1), A3, Z);
  if (e == cudaSuccess) e = lincomb(c, A3, 1.0, A3, 0, nullptr, 0, nullptr, 1.0, dt_dev, Z);    /* Ubar1 */
  /* stage 1: U1 = U^n + dt L(U^n) */
  if (e == cudaSuccess) e = adj_sweeps(c, U_n, F(0), Lz(0), A3, Z);
  if (e == cudaSuccess)
    e = lincomb(c, Ubar_n, 1.0 / 3.0, Ubar_np1, 0.75, A2, 1.0, A3, 1.0, dt_dev, Z);
  return e == cudaSuccess ? TENOM_OK : cuda_fail(c, e, "rk3_step_adjoint");
}

tenom_status tenom_rk3_step_adjoint_tape(tenom_ctx* c, const double* U_n, const double* tape_states,
                                         const uint8_t* tape_flags, const double* dt_dev, const double* Ubar_np1,
                                         double* Ubar_n) {
  if (!c) return TENOM_E_INVALID;
  if (!aligned8(U_n) || !aligned8(tape_states) || !tape_flags || !aligned8(dt_dev) || !aligned8(Ubar_np1) ||
      !aligned8(Ubar_n) || Ubar_n == Ubar_np1)
    return fail(c, TENOM_E_INVALID, "rk3_step_adjoint: bad pointers");
  return adjoint_step(c, U_n, tape_states, tape_flags, nullptr, dt_dev, Ubar_np1, Ubar_n);
}

tenom_status tenom_rk3_step_adjoint_lin(tenom_ctx* c, const double* U_n, const double* tape_states,
                                        const double* tape_lin, const double* dt_dev, const double* Ubar_np1,
                                        double* Ubar_n) {
  if (!c) return TENOM_E_INVALID;
  if (!aligned8(U_n) || !aligned8(tape_states) || !aligned8(tape_lin) || !aligned8(dt_dev) || !aligned8(Ubar_np1) ||
      !aligned8(Ubar_n) || Ubar_n == Ubar_np1)
    return fail(c, TENOM_E_INVALID, "rk3_step_adjoint_lin: bad pointers");
  return adjoint_step(c, U_n, tape_states, nullptr, tape_lin, dt_dev, Ubar_np1, Ubar_n);
}

tenom_status tenom_rk3_step_adjoint(tenom_ctx* c, const double* U_n, const double* dt_dev, const double* Ubar_np1,
                                    double* Ubar_n) {
  if (!c) return TENOM_E_INVALID;
  if (adjoint_unsupported(c, "rk3_step_adjoint")) return TENOM_E_UNSUPPORTED;
  if (!aligned8(U_n) || !aligned8(dt_dev)) return fail(c, TENOM_E_INVALID, "rk3_step_adjoint: bad pointers");
  cudaError_t e = ensure_adj(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "rk3_step_adjoint");
  const long long n = c->nv * c->ncell;
  double* Uc = c->adj + 4 * n;  /* copy of U^n advanced by the recording step */
  e = cudaMemcpyAsync(Uc, U_n, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess && dt_dev != c->dt)
    e = cudaMemcpyAsync(c->dt, dt_dev, sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  if (e == cudaSuccess) e = rk3_record(c, Uc, c->adj + 5 * n, c->adj + 6 * n, c->adj_flags, nullptr);
  if (e != cudaSuccess) return cuda_fail(c, e, "rk3_step_adjoint");
  return tenom_rk3_step_adjoint_tape(c, U_n, c->adj + 5 * n, c->adj_flags, dt_dev, Ubar_np1, Ubar_n);
}

tenom_status tenom_check_fastmath(const double* x, double* out, long long n, void* stream) {
  if (!x || !out || n < 0) return TENOM_E_INVALID;
  fastmath_check_kernel<<<ew_blocks(n), 256, 0, (cudaStream_t)stream>>>(x, out, n);
  return cudaGetLastError() == cudaSuccess ? TENOM_OK : TENOM_E_CUDA;
}

tenom_status tenom_fp64_peak(void* stream, int nblocks, int iters, double* flops) {
  if (nblocks < 1 || iters < 1 || !flops) return TENOM_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  double* sink = nullptr;
  cudaEvent_t a, b;
  cudaError_t e = cudaMalloc(&sink, sizeof(double));
  if (e != cudaSuccess) return TENOM_E_CUDA;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  dfma_probe_kernel<<<nblocks, 256, 0, st>>>(iters / 8 + 1, 0.999999, 1e-7, sink);  /* warm-up */
  cudaEventRecord(a, st);
  dfma_probe_kernel<<<nblocks, 256, 0, st>>>(iters, 0.999999, 1e-7, sink);
  cudaEventRecord(b, st);
  e = cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (e != cudaSuccess) return TENOM_E_CUDA;
  *flops = 2.0 * 8.0 * (double)iters * nblocks * 256.0 / (ms * 1e-3);
  return TENOM_OK;
}

}  // extern "C"

/* ---------------------------------------------------------------- helpers for other units */
namespace tenom {

tenom_status check_grid_scheme(const tenom_grid* g, const tenom_scheme* s, std::string* msg) {
  return validate(g, s, msg);
}

SchemeDev scheme_for_device(const tenom_scheme& s) {
  tenom_scheme t = s;
  bool anyd = false;
  for (int k = 0; k < 6; ++k) anyd |= (t.d[k] != 0.0);
  if (!anyd)
    for (int k = 0; k < t.K - 2; ++k) t.d[k] = (t.K == 6) ? kDopt6[k] : kDopt8[k];
  return scheme_dev(t);
}

cudaError_t launch_rhs_divergence(int nv, double* const F[3], const int n[3], const double dx[3], long long ncell,
                                  const long long nface[3], double* out, cudaStream_t st) {
  StageArgs a;
  memset(&a, 0, sizeof(a));
  for (int d = 0; d < 3; ++d) {
    a.cu.F[d] = F[d];
    a.n[d] = n[d];
    a.cu.rdx[d] = 1.0 / dx[d];
    a.cu.nface[d] = nface[d];
  }
  a.cu.out = out;
  a.ncell = ncell;
  a.cu.mode = 0;
  return launch_stage_kernel(nv, a, st);
}

}  // namespace tenom
