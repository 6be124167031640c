/* The batched SSP-RK3 stage kernel (see tenom_batch.cu), shared by the translation units
   that instantiate it: tenom_batch.cu (without the positivity limiter) and
   tenom_batch_pp.cu (with it). */
#pragma once
#include "tenom_internal.h"
#include "tenom_positivity.cuh"

namespace tenom {

struct BatchArgs {
  const int* n;
  const long long* off;
  const double* dx;
  const int* bc;
  const double* dt;
  const int2* items;
  int nitems;
  int* counter;
  int* status;
  long long total;
  double gamma;
  SchemeDev sch;
};

template <int K, int TILE>
struct BatchTile {
  static constexpr int NV = 3;
  static constexpr int NP = TILE + K - 1;
  static constexpr size_t SMEM = sizeof(double) * (PointLayout<3>::NC * NP + NV * TILE);
};

/* stage: 1 -> out = Us + dt L(Us); 2,3 -> out = cA U0 + cB (Us + dt L(Us)).  Compiled for
   512 resident threads per SM (128 registers a thread), so that the autotuner's CTA counts
   can reach 16 warps per SM. */
template <int K, int LIM, int TILE, bool PP>
__global__ void __launch_bounds__(TILE, 512 / TILE)
batch_stage_kernel(const BatchArgs A, const double* __restrict__ Us, const double* __restrict__ U0, double* out,
                   int mode, double cA, double cB) {
  using T = BatchTile<K, TILE>;
  constexpr int NV = 3, H = K / 2, NP = T::NP;
  extern __shared__ double sm[];
  double* Fs = sm + PointLayout<3>::NC * NP;
  __shared__ int s_item;
  const int tid = threadIdx.x;
  int st = 0;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(A.counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= A.nitems) break;
    const int2 w = A.items[it];
    const int j = w.x, f0 = w.y;
    const double dt = A.dt[j];
    if (dt == 0.0) continue;  /* finished problem (uniform across the CTA) */
    const int n = A.n[j];
    const long long off = A.off[j];
    const int bc = A.bc[j];
    for (int p = tid; p < NP; p += TILE) {
      const int jj = bc_wrap(f0 - H + p, n, bc);
      double u[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) u[q] = Us[q * A.total + off + jj];
      stage_point<NV, 0>(u, A.gamma, sm, NP, p, st);
    }
    __syncthreads();
    if (f0 + tid <= n) {
      double Fh[NV];
      face_flux_smem<NV, K, LIM, 0, 1>(sm, NP, tid, 0, A.gamma, A.sch, Fh, nullptr, st);
      if constexpr (PP) {
        /* positivity limiter of this stage (length dt, 1D: mu = 2 dt/dx) on the face between
           staged points tid + H - 1 and tid + H; a face computed by two items is limited
           identically by both */
        using L = PointLayout<NV>;
        const double mu = 2.0 * dt / A.dx[j];
        double Ua[NV], Ub[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          Ua[v] = sm[(L::cU + v) * NP + tid + H - 1];
          Ub[v] = sm[(L::cU + v) * NP + tid + H];
        }
        positivity_face<NV, 0>(Ua, Ub, Fh, mu, A.gamma, f32_rz(mu), f32_rz(A.gamma - 1.0));
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) Fs[v * TILE + tid] = Fh[v];
    }
    __syncthreads();
    const int c = f0 + tid;
    if (tid < TILE - 1 && c < n) {
      const double dxj = A.dx[j];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double r = 0.0 - (Fs[v * TILE + tid + 1] - Fs[v * TILE + tid]) / dxj;
        const long long g = v * A.total + off + c;
        const double t1 = Us[g] + dt * r;
        out[g] = (mode == 1) ? t1 : cA * U0[g] + cB * t1;
      }
    }
    __syncthreads();
  }
  if (st) atomicOr(A.status, st);
}

using StageFn = void (*)(const BatchArgs, const double*, const double*, double*, int, double, double);

/* stage kernels with the positivity limiter, for K in {6, 8}, LIM in {MP, TVD5},
   TILE in {64, 128, 256} (tenom_batch_pp.cu); null for other combinations */
StageFn pick_stage_pp(int K, int lim, int tile);

}  // namespace tenom
