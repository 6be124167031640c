/* tenom_rhs_noalloc: the operator dU/dt = L(U) of tenom_rhs for callers that cannot
 * allocate device memory (see include/tenom.h).  Its scratch -- the face-flux buffers of
 * every axis and a status word -- lives in one file-scope device array, so a call needs no
 * context and performs no allocation.  Every GPU that loads this library holds the array
 * (TENOM_NOALLOC_SCRATCH_BYTES) until the process exits. */
#include <cstdio>
#include <mutex>
#include <string>

#include "tenom.h"
#include "tenom_internal.h"

namespace tenom {

/* first 256 bytes: status word; then the face buffers, axis after axis */
static __device__ __align__(256) double g_noalloc_scratch[TENOM_NOALLOC_SCRATCH_BYTES / sizeof(double)];

static constexpr long long kStatusDoubles = 256 / sizeof(double);
static constexpr int kMaxDevices = 64;
static std::mutex g_setup_mu;
static double* g_scratch_dev[kMaxDevices];  /* device address of the array, per device */

/* Once per device, with that device current: look up the array's device address.  In
 * host code the symbol g_noalloc_scratch is only a host-side stand-in and must never be
 * handed to a kernel. */
static cudaError_t scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

}  // namespace tenom

using namespace tenom;

extern "C" tenom_status tenom_rhs_noalloc(const tenom_grid* grid, const tenom_scheme* scheme, const double* U,
                                          double* dUdt, int* status_dev, void* stream) {
  std::string msg;
  tenom_status v = check_grid_scheme(grid, scheme, &msg);
  if (v != TENOM_OK) {
    fprintf(stderr, "tenom_rhs_noalloc: %s\n", msg.c_str());
    return v;
  }
  if (!U || !dUdt || ((uintptr_t)U & 7) || ((uintptr_t)dUdt & 7) || U == dUdt ||
      ((uintptr_t)status_dev & 3)) {
    fprintf(stderr, "tenom_rhs_noalloc: bad pointers\n");
    return TENOM_E_INVALID;
  }
  const int nv = grid->dim + 2;
  const long long ncell = (long long)grid->n[0] * grid->n[1] * grid->n[2];
  long long nface[3] = {0, 0, 0};
  long long need = kStatusDoubles;
  for (int a = 0; a < grid->dim; ++a) {
    nface[a] = ncell / grid->n[a] * (grid->n[a] + 1);
    need += nv * nface[a];
  }
  const long long cap = (long long)(TENOM_NOALLOC_SCRATCH_BYTES / sizeof(double));
  if (need > cap) {
    fprintf(stderr,
            "tenom_rhs_noalloc: grid needs %lld bytes of face scratch, the static scratch holds %lld "
            "(use tenom_create/tenom_rhs for this grid)\n",
            need * (long long)sizeof(double), cap * (long long)sizeof(double));
    return TENOM_E_INVALID;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    fprintf(stderr, "tenom_rhs_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
    return TENOM_E_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* status = status_dev ? status_dev : reinterpret_cast<int*>(scratch);
  if (!status_dev) {
    e = cudaMemsetAsync(status, 0, sizeof(int), st);  /* the shared word keeps the last call's bits */
    if (e != cudaSuccess) return TENOM_E_CUDA;
  }
  double* F[3] = {nullptr, nullptr, nullptr};
  long long off = kStatusDoubles;
  for (int a = 0; a < grid->dim; ++a) {
    F[a] = scratch + off;
    off += nv * nface[a];
  }
  FaceArgs fa;
  memset(&fa, 0, sizeof(fa));
  fa.U = U;
  fa.flags = nullptr;
  fa.status = status;
  for (int d = 0; d < 3; ++d) {
    fa.n[d] = grid->n[d];
    fa.bc[d] = grid->bc[d];
  }
  fa.ncell = ncell;
  fa.gamma = grid->gamma;
  fa.sch = scheme_for_device(*scheme);
  for (int a = 0; a < grid->dim && e == cudaSuccess; ++a) {
    fa.Fhat = F[a];
    fa.nface = nface[a];
    if (nv == 3) e = launch_face_nv3(fa, a, scheme->K, scheme->limiter, st);
    else if (nv == 4) e = launch_face_nv4(fa, a, scheme->K, scheme->limiter, st);
    else e = launch_face_nv5(fa, a, scheme->K, scheme->limiter, st);
  }
  if (e == cudaSuccess) e = launch_rhs_divergence(nv, F, grid->n, grid->dx, ncell, nface, dUdt, st);
  if (e != cudaSuccess) {
    fprintf(stderr, "tenom_rhs_noalloc: %s\n", cudaGetErrorString(e));
    return TENOM_E_CUDA;
  }
  return TENOM_OK;
}
