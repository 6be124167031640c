/* Batched solver: many independent 1D Euler problems of uneven size advanced together.
 *
 * State: one concatenated array U[3][total]; problem j owns cells [off_j, off_j + n_j).
 * Each SSP-RK3 stage is ONE persistent kernel: CTAs take work items (problem j, first face
 * f0) from a global counter; an item stages TILE + K - 1 points, computes the TILE faces
 * f0 .. f0 + TILE - 1 of problem j (the same device code as the single-grid solver), then
 * updates the TILE - 1 cells whose two faces it owns (flux difference + stage combine).
 * Consecutive items of a problem overlap by one face, which is computed twice, so no CTA
 * ever waits for another (no grid barrier).  Per-problem time steps come from a per-problem
 * CFL reduction; a finished problem (t_j >= t_end_j) has dt_j = 0 and its items are skipped,
 * which leaves its state untouched.  One RK3 step (CFL reduction, dt, three stage kernels,
 * time update) is captured once into a CUDA graph and replayed.  The tile size and the
 * number of resident CTAs per SM are chosen by timing the candidates on the actual batch
 * (tenom_batch_autotune). */
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tenom.h"
#include "tenom_internal.h"
#include "tenom_batch_kernel.cuh"

namespace tenom {

/* per-problem max_i (|u| + c)_i / dx over cell tiles (problem, first cell) of 256 cells */
__global__ void batch_signal_kernel(const double* __restrict__ U, long long total, const int2* citems, const int* n,
                                    const long long* off, const double* dx, double gamma, const double* dt_prev,
                                    unsigned long long* smax, int* status) {
  const int2 w = citems[blockIdx.x];
  const int j = w.x;
  const int c = w.y + threadIdx.x;
  double s = 0.0;
  int st = 0;
  if (c < n[j]) {
    const long long g = off[j] + c;
    const double rho = U[g], m = U[total + g], E = U[2 * total + g];
    const double u = m / rho;
    const double p = (gamma - 1.0) * (E - 0.5 * (m * u));
    if (!(rho > 0.0)) st |= ST_RHO;
    if (!(p > 0.0)) st |= ST_P;
    const double cs = sqrt(gamma * p / rho);
    s = (fabs(u) + cs) / dx[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, s, o);
    s = t > s ? t : s;
  }
  __shared__ double red[8];
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[wi] = s;
  __syncthreads();
  if (wi == 0) {
    s = (l < 8) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_xor_sync(0xffffffffu, s, o);
      s = t > s ? t : s;
    }
    if (l == 0 && s == s) atomicMax(smax + j, (unsigned long long)__double_as_longlong(s));
  }
  if (st) atomicOr(status, st);
}

/* dt_j = min(cfl / smax_j, t_end_j - t_j), 0 once t_j >= t_end_j; resets smax_j */
__global__ void batch_finalize_kernel(int P, unsigned long long* smax, double cfl, const double* t, const double* t_end,
                                      double* dt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  const double s = __longlong_as_double((long long)smax[j]);
  const double rem = t_end[j] - t[j];
  double d = cfl / s;
  d = rem < d ? rem : d;
  dt[j] = (rem > 0.0) ? d : 0.0;
  smax[j] = 0ull;
}

__global__ void batch_time_kernel(int P, double* t, const double* dt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < P) t[j] = t[j] + dt[j];
}

__global__ void batch_init_kernel(const double* prim, double* U, long long total, double gamma) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total; c += (long long)gridDim.x * blockDim.x) {
    const double rho = prim[c], u = prim[total + c], p = prim[2 * total + c];
    U[c] = rho;
    U[total + c] = rho * u;
    U[2 * total + c] = p / (gamma - 1.0) + 0.5 * (rho * u * u);
  }
}

template <int K, int LIM, int TILE>
static StageFn stage_fn() { return batch_stage_kernel<K, LIM, TILE, false>; }

static StageFn pick_stage(int K, int lim, int tile, bool pp) {
  if (pp) return pick_stage_pp(K, lim, tile);
#define TENOM_PICK(KK, LL, TT) if (K == KK && lim == LL && tile == TT) return stage_fn<KK, LL, TT>();
  TENOM_PICK(6, LIM_MP, 64) TENOM_PICK(6, LIM_MP, 128) TENOM_PICK(6, LIM_MP, 256)
  TENOM_PICK(6, LIM_TVD5, 64) TENOM_PICK(6, LIM_TVD5, 128) TENOM_PICK(6, LIM_TVD5, 256)
  TENOM_PICK(8, LIM_MP, 64) TENOM_PICK(8, LIM_MP, 128) TENOM_PICK(8, LIM_MP, 256)
  TENOM_PICK(8, LIM_TVD5, 64) TENOM_PICK(8, LIM_TVD5, 128) TENOM_PICK(8, LIM_TVD5, 256)
#undef TENOM_PICK
  return nullptr;
}

/* dynamic shared memory of the stage kernel of (K, tile): the kernel's own layout */
static size_t stage_smem(int K, int tile) {
  if (K == 6) return tile == 64 ? BatchTile<6, 64>::SMEM : (tile == 128 ? BatchTile<6, 128>::SMEM : BatchTile<6, 256>::SMEM);
  return tile == 64 ? BatchTile<8, 64>::SMEM : (tile == 128 ? BatchTile<8, 128>::SMEM : BatchTile<8, 256>::SMEM);
}

}  // namespace tenom

using namespace tenom;

struct tenom_batch {
  int P;
  long long total;
  tenom_scheme s;
  double gamma;
  cudaStream_t st;      /* caller's stream */
  cudaStream_t cap;     /* internal stream used for graph capture */
  int sms;
  /* device */
  int* n_d;
  long long* off_d;
  double* dx_d;
  int* bc_d;
  double* t_d;
  double* tend_d;
  double* dt_d;
  unsigned long long* smax_d;
  int* counters_d;      /* 3 stage counters + status */
  int* status_d;
  int2* items_d;
  int nitems;
  int2* citems_d;
  int ncitems;
  double* W1;
  double* W2;
  /* host */
  std::vector<int> n;
  std::vector<long long> off;
  int tile;
  int ctas_per_sm;
  /* graph */
  cudaGraphExec_t exec;
  const double* graph_U;
  double graph_cfl;
  std::string err;
};

static tenom_status bfail(tenom_batch* b, tenom_status s, const std::string& m) {
  if (b) b->err = m;
  fprintf(stderr, "tenom_batch: %s\n", m.c_str());
  return s;
}

static cudaError_t build_items(tenom_batch* b, int tile) {
  std::vector<int2> items;
  std::vector<int> order(b->P);
  for (int j = 0; j < b->P; ++j) order[j] = j;
  std::sort(order.begin(), order.end(), [&](int a, int c) { return b->n[a] > b->n[c]; });
  for (int j : order)
    for (int f0 = 0; f0 < b->n[j]; f0 += tile - 1) items.push_back(make_int2(j, f0));
  cudaFree(b->items_d);
  b->items_d = nullptr;
  b->nitems = (int)items.size();
  cudaError_t e = cudaMalloc(&b->items_d, sizeof(int2) * items.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->items_d, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  b->tile = tile;
  /* shared-memory size of the stage kernel for this tile (set outside any graph capture) */
  StageFn fn = pick_stage(b->s.K, b->s.limiter, tile, b->s.positivity == TENOM_PP_ON);
  if (e == cudaSuccess && fn)
    e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)stage_smem(b->s.K, tile));
  return e;
}

static BatchArgs batch_args(tenom_batch* b, int stage) {
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.n = b->n_d;
  a.off = b->off_d;
  a.dx = b->dx_d;
  a.bc = b->bc_d;
  a.dt = b->dt_d;
  a.items = b->items_d;
  a.nitems = b->nitems;
  a.counter = b->counters_d + (stage - 1);
  a.status = b->status_d;
  a.total = b->total;
  a.gamma = b->gamma;
  a.sch = scheme_for_device(b->s);
  return a;
}

static cudaError_t launch_stage_b(tenom_batch* b, int stage, double* U, cudaStream_t st) {
  StageFn fn = pick_stage(b->s.K, b->s.limiter, b->tile, b->s.positivity == TENOM_PP_ON);
  if (!fn) return cudaErrorNotSupported;
  const size_t smem = stage_smem(b->s.K, b->tile);
  BatchArgs a = batch_args(b, stage);
  const int grid = std::max(1, std::min(b->nitems, b->sms * b->ctas_per_sm));
  const double* Us = (stage == 1) ? U : (stage == 2 ? b->W1 : b->W2);
  double* out = (stage == 1) ? b->W1 : (stage == 2 ? b->W2 : U);
  const int mode = (stage == 1) ? 1 : 2;
  const double cA = (stage == 2) ? 0.75 : 1.0 / 3.0, cB = (stage == 2) ? 0.25 : 2.0 / 3.0;
  fn<<<grid, b->tile, smem, st>>>(a, Us, U, out, mode, cA, cB);
  return cudaGetLastError();
}

static cudaError_t record_step(tenom_batch* b, double* U, double cfl, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->counters_d, 0, sizeof(int) * 3, st);
  if (e != cudaSuccess) return e;
  batch_signal_kernel<<<b->ncitems, 256, 0, st>>>(U, b->total, b->citems_d, b->n_d, b->off_d, b->dx_d, b->gamma,
                                                   b->dt_d, b->smax_d, b->status_d);
  batch_finalize_kernel<<<(b->P + 127) / 128, 128, 0, st>>>(b->P, b->smax_d, cfl, b->t_d, b->tend_d, b->dt_d);
  e = cudaGetLastError();
  for (int s = 1; s <= 3 && e == cudaSuccess; ++s) e = launch_stage_b(b, s, U, st);
  if (e == cudaSuccess) {
    batch_time_kernel<<<(b->P + 127) / 128, 128, 0, st>>>(b->P, b->t_d, b->dt_d);
    e = cudaGetLastError();
  }
  return e;
}

static void drop_graph(tenom_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->graph_U = nullptr;
}

extern "C" {

tenom_status tenom_batch_create(tenom_batch** out, int nprob, const int* n, const double* dx, const int* bc, double gamma,
                                const tenom_scheme* scheme, void* stream) {
  if (!out) return TENOM_E_INVALID;
  *out = nullptr;
  if (nprob < 1 || !n || !dx || !scheme || !(gamma > 1.0)) return bfail(nullptr, TENOM_E_INVALID, "bad arguments");
  if (scheme->K != 6 && scheme->K != 8) return bfail(nullptr, TENOM_E_INVALID, "K must be 6 or 8");
  if (scheme->limiter != TENOM_LIM_MP && scheme->limiter != TENOM_LIM_TVD5)
    return bfail(nullptr, TENOM_E_UNSUPPORTED, "limiter not built");
  if (scheme->positivity != TENOM_PP_OFF && scheme->positivity != TENOM_PP_ON)
    return bfail(nullptr, TENOM_E_INVALID, "bad positivity flag");
  tenom_batch* b = new tenom_batch();
  b->P = nprob;
  b->s = *scheme;
  b->gamma = gamma;
  b->st = (cudaStream_t)stream;
  b->exec = nullptr;
  b->graph_U = nullptr;
  b->n.assign(n, n + nprob);
  b->off.resize(nprob + 1);
  std::vector<int> bch(nprob, TENOM_BC_TRANSMISSIVE);
  long long tot = 0;
  for (int j = 0; j < nprob; ++j) {
    if (n[j] < 1 || n[j] > (1 << 24) || !(dx[j] > 0.0)) {
      delete b;
      return bfail(nullptr, TENOM_E_INVALID, "bad problem size or spacing");
    }
    if (bc) bch[j] = bc[j];
    if (bch[j] != TENOM_BC_PERIODIC && bch[j] != TENOM_BC_TRANSMISSIVE) {
      delete b;
      return bfail(nullptr, TENOM_E_INVALID, "bad bc");
    }
    if (bch[j] == TENOM_BC_PERIODIC && n[j] < scheme->K / 2) {
      delete b;
      return bfail(nullptr, TENOM_E_INVALID, "periodic problem shorter than the half stencil");
    }
    b->off[j] = tot;
    tot += n[j];
  }
  b->off[nprob] = tot;
  b->total = tot;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  std::vector<int2> citems;
  for (int j = 0; j < nprob; ++j)
    for (int c0 = 0; c0 < n[j]; c0 += 256) citems.push_back(make_int2(j, c0));
  b->ncitems = (int)citems.size();
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  A((void**)&b->n_d, sizeof(int) * nprob);
  A((void**)&b->off_d, sizeof(long long) * nprob);
  A((void**)&b->dx_d, sizeof(double) * nprob);
  A((void**)&b->bc_d, sizeof(int) * nprob);
  A((void**)&b->t_d, sizeof(double) * nprob);
  A((void**)&b->tend_d, sizeof(double) * nprob);
  A((void**)&b->dt_d, sizeof(double) * nprob);
  A((void**)&b->smax_d, sizeof(unsigned long long) * nprob);
  A((void**)&b->counters_d, sizeof(int) * 4);
  A((void**)&b->citems_d, sizeof(int2) * citems.size());
  A((void**)&b->W1, sizeof(double) * 3 * tot);
  A((void**)&b->W2, sizeof(double) * 3 * tot);
  if (e == cudaSuccess) {
    b->status_d = b->counters_d + 3;
    std::vector<double> zero(nprob, 0.0), inf(nprob, HUGE_VAL);
    e = cudaMemcpy(b->n_d, n, sizeof(int) * nprob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->off_d, b->off.data(), sizeof(long long) * nprob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->dx_d, dx, sizeof(double) * nprob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->bc_d, bch.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->t_d, zero.data(), sizeof(double) * nprob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->tend_d, inf.data(), sizeof(double) * nprob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->smax_d, 0, sizeof(unsigned long long) * nprob);
    if (e == cudaSuccess) e = cudaMemset(b->counters_d, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(b->dt_d, 0, sizeof(double) * nprob);
    if (e == cudaSuccess)
      e = cudaMemcpy(b->citems_d, citems.data(), sizeof(int2) * citems.size(), cudaMemcpyHostToDevice);
  }
  b->ctas_per_sm = 2;
  if (e == cudaSuccess) e = build_items(b, 128);
  if (e != cudaSuccess) {
    std::string m = cudaGetErrorString(e);
    tenom_batch_destroy(b);
    return bfail(nullptr, TENOM_E_CUDA, m);
  }
  *out = b;
  return TENOM_OK;
}

tenom_status tenom_batch_destroy(tenom_batch* b) {
  if (!b) return TENOM_OK;
  cudaStreamSynchronize(b->st);
  drop_graph(b);
  void* ps[] = {b->n_d, b->off_d, b->dx_d, b->bc_d, b->t_d, b->tend_d, b->dt_d, b->smax_d,
                b->counters_d, b->items_d, b->citems_d, b->W1, b->W2};
  for (void* p : ps) cudaFree(p);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return TENOM_OK;
}

tenom_status tenom_batch_layout(const tenom_batch* b, long long* off_host, long long* total) {
  if (!b || !off_host || !total) return TENOM_E_INVALID;
  for (int j = 0; j <= b->P; ++j) off_host[j] = b->off[j];
  *total = b->total;
  return TENOM_OK;
}

tenom_status tenom_batch_init_state(tenom_batch* b, const double* prim, double* U) {
  if (!b || !prim || !U || prim == U) return TENOM_E_INVALID;
  long long nb = (b->total + 255) / 256;
  batch_init_kernel<<<(unsigned)std::min<long long>(nb, 152 * 16), 256, 0, b->st>>>(prim, U, b->total, b->gamma);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TENOM_OK : bfail(b, TENOM_E_CUDA, cudaGetErrorString(e));
}

tenom_status tenom_batch_set_time(tenom_batch* b, const double* t_host, const double* t_end_host) {
  if (!b) return TENOM_E_INVALID;
  cudaError_t e = cudaSuccess;
  if (t_host) e = cudaMemcpyAsync(b->t_d, t_host, sizeof(double) * b->P, cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess && t_end_host)
    e = cudaMemcpyAsync(b->tend_d, t_end_host, sizeof(double) * b->P, cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  return e == cudaSuccess ? TENOM_OK : bfail(b, TENOM_E_CUDA, cudaGetErrorString(e));
}

tenom_status tenom_batch_get_time(tenom_batch* b, double* t_host) {
  if (!b || !t_host) return TENOM_E_INVALID;
  cudaError_t e = cudaMemcpyAsync(t_host, b->t_d, sizeof(double) * b->P, cudaMemcpyDeviceToHost, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  return e == cudaSuccess ? TENOM_OK : bfail(b, TENOM_E_CUDA, cudaGetErrorString(e));
}

tenom_status tenom_batch_status_word(tenom_batch* b, int* status_host, int reset) {
  if (!b || !status_host) return TENOM_E_INVALID;
  cudaError_t e = cudaMemcpyAsync(status_host, b->status_d, sizeof(int), cudaMemcpyDeviceToHost, b->st);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(b->status_d, 0, sizeof(int), b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return bfail(b, TENOM_E_CUDA, cudaGetErrorString(e));
  return *status_host ? TENOM_E_NONPHYSICAL : TENOM_OK;
}

tenom_status tenom_batch_stage(tenom_batch* b, int stage, double* U) {
  if (!b || !U || stage < 1 || stage > 3) return TENOM_E_INVALID;
  cudaError_t e = cudaMemsetAsync(b->counters_d + (stage - 1), 0, sizeof(int), b->st);
  if (e == cudaSuccess) e = launch_stage_b(b, stage, U, b->st);
  return e == cudaSuccess ? TENOM_OK : bfail(b, TENOM_E_CUDA, cudaGetErrorString(e));
}

tenom_status tenom_batch_step(tenom_batch* b, double* U, double cfl, int nsteps) {
  if (!b || !U || !(cfl > 0.0) || nsteps < 0) return TENOM_E_INVALID;
  cudaError_t e = cudaSuccess;
  if (!b->exec || b->graph_U != U || b->graph_cfl != cfl) {
    drop_graph(b);
    /* capture on the internal stream (the caller's may be the legacy default stream) */
    cudaGraph_t g = nullptr;
    e = cudaStreamSynchronize(b->st);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t er = record_step(b, U, cfl, b->cap);
      e = cudaStreamEndCapture(b->cap, &g);
      if (er != cudaSuccess) e = er;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, TENOM_E_CUDA, std::string("graph: ") + cudaGetErrorString(e));
    b->graph_U = U;
    b->graph_cfl = cfl;
  }
  for (int k = 0; k < nsteps && e == cudaSuccess; ++k) e = cudaGraphLaunch(b->exec, b->st);
  return e == cudaSuccess ? TENOM_OK : bfail(b, TENOM_E_CUDA, cudaGetErrorString(e));
}

tenom_status tenom_batch_step_direct(tenom_batch* b, double* U, double cfl, int nsteps) {
  if (!b || !U || !(cfl > 0.0) || nsteps < 0) return TENOM_E_INVALID;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < nsteps && e == cudaSuccess; ++k) e = record_step(b, U, cfl, b->st);
  return e == cudaSuccess ? TENOM_OK : bfail(b, TENOM_E_CUDA, cudaGetErrorString(e));
}

tenom_status tenom_batch_autotune(tenom_batch* b, double* U, int* tile_out, int* ctas_out) {
  if (!b || !U) return TENOM_E_INVALID;
  const int tiles[3] = {64, 128, 256};
  const int ctas[4] = {1, 2, 4, 8};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  /* a first stage-1 launch needs dt: compute it once (no time update) */
  cudaError_t e = cudaMemsetAsync(b->counters_d, 0, sizeof(int) * 3, b->st);
  batch_signal_kernel<<<b->ncitems, 256, 0, b->st>>>(U, b->total, b->citems_d, b->n_d, b->off_d, b->dx_d, b->gamma,
                                                     b->dt_d, b->smax_d, b->status_d);
  batch_finalize_kernel<<<(b->P + 127) / 128, 128, 0, b->st>>>(b->P, b->smax_d, 0.4, b->t_d, b->tend_d, b->dt_d);
  float best = 1e30f;
  int bt = b->tile, bc = b->ctas_per_sm;
  for (int ti = 0; ti < 3 && e == cudaSuccess; ++ti) {
    e = build_items(b, tiles[ti]);
    StageFn fn = pick_stage(b->s.K, b->s.limiter, tiles[ti], b->s.positivity == TENOM_PP_ON);
    int occ = 0;
    const size_t smem = stage_smem(b->s.K, tiles[ti]);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn, tiles[ti], smem);
    for (int ci = 0; ci < 4 && e == cudaSuccess; ++ci) {
      if (ctas[ci] > occ) continue;
      b->ctas_per_sm = ctas[ci];
      float ms_best = 1e30f;
      for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        e = cudaMemsetAsync(b->counters_d, 0, sizeof(int), b->st);
        cudaEventRecord(e0, b->st);
        if (e == cudaSuccess) e = launch_stage_b(b, 1, U, b->st);
        cudaEventRecord(e1, b->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) ms_best = std::min(ms_best, ms);
      }
      if (ms_best < best) {
        best = ms_best;
        bt = tiles[ti];
        bc = ctas[ci];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = build_items(b, bt);
  b->ctas_per_sm = bc;
  drop_graph(b);
  if (e != cudaSuccess) return bfail(b, TENOM_E_CUDA, cudaGetErrorString(e));
  if (tile_out) *tile_out = bt;
  if (ctas_out) *ctas_out = bc;
  return TENOM_OK;
}

tenom_status tenom_batch_set_tiling(tenom_batch* b, int tile, int ctas_per_sm) {
  if (!b || (tile != 64 && tile != 128 && tile != 256) || ctas_per_sm < 1 || ctas_per_sm > 16)
    return TENOM_E_INVALID;
  b->ctas_per_sm = ctas_per_sm;
  drop_graph(b);
  cudaError_t e = build_items(b, tile);
  return e == cudaSuccess ? TENOM_OK : bfail(b, TENOM_E_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
