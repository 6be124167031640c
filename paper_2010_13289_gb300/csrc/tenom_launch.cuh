/* Host-side launchers of the face sweeps and their adjoints, templated on the Euler system (NV = 3, 4, 5 for
 * 1D, 2D, 3D); each tenom_*_nvN.cu file instantiates one NV so the kernels compile in
 * parallel.  Dynamic shared memory above 48 KB is opted into once per kernel and device:
 * the attribute belongs to the device's context, so a process that launches on a second
 * GPU sets it there too. */
#pragma once
#include <atomic>
#include <mutex>
#include "tenom_internal.h"
#include "tenom_adjoint_kernels.cuh"

namespace tenom {

/* Per kernel: whether its shared-memory attribute has been set on each device.  Readers
   take the flag without the lock; the first launch on a device sets the attribute under
   the lock and only then publishes the flag. */
struct AttrOnce {
  static constexpr int kMaxDevices = 64;
  std::atomic<bool> done[kMaxDevices];
  std::mutex mu;
  AttrOnce() {
    for (auto& d : done) d.store(false, std::memory_order_relaxed);
  }
};

template <class Kern>
static cudaError_t ensure_smem_attr(Kern kern, AttrOnce& attr, size_t smem) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= AttrOnce::kMaxDevices) return cudaErrorInvalidDevice;
  if (attr.done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(attr.mu);
  if (attr.done[dev].load(std::memory_order_relaxed)) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  attr.done[dev].store(true, std::memory_order_release);
  return cudaSuccess;
}

template <class Kern>
static cudaError_t launch_tile(Kern kern, AttrOnce& attr, size_t smem, int nv, int axis, const int* n, int K,
                               cudaStream_t st, const void* args_ptr, bool wrapped = false,
                               bool fwd_tile = false) {
  cudaError_t e = ensure_smem_attr(kern, attr, smem);
  if (e != cudaSuccess) return e;
  dim3 grid, block;
  face_grid(nv, axis, n, K, &grid, &block, wrapped, fwd_tile);
  void* argv[1] = {const_cast<void*>(args_ptr)};
  return cudaLaunchKernel((const void*)kern, grid, block, argv, smem, st);
}

/* forward face sweep (REC: also record the linearisation; STATS: decision statistics
   instead of fluxes) */
template <int NV, int K, int LIM, int AXIS, bool REC, bool STATS>
static cudaError_t launch_face_one(const FaceArgs& a, cudaStream_t st) {
  static AttrOnce attr;
  return launch_tile(face_kernel<NV, K, LIM, AXIS, REC, STATS>, attr, face_smem<NV, K, AXIS, REC, STATS>(), NV, AXIS,
                     a.n, K, st, &a, !STATS && a.bc[AXIS] == 0, !STATS);
}

template <int NV, int AXIS, bool REC, bool STATS>
static cudaError_t launch_face_axis(const FaceArgs& a, int K, int lim, cudaStream_t st) {
  if (K == 6) {
    if (lim == LIM_MP) return launch_face_one<NV, 6, LIM_MP, AXIS, REC, STATS>(a, st);
    if (lim == LIM_TVD5) return launch_face_one<NV, 6, LIM_TVD5, AXIS, REC, STATS>(a, st);
    if constexpr (!REC)  /* Van Albada: forward only (no frozen linear form to record) */
      if (lim == LIM_VA) return launch_face_one<NV, 6, LIM_VA, AXIS, false, STATS>(a, st);
  } else if (K == 8) {
    if (lim == LIM_MP) return launch_face_one<NV, 8, LIM_MP, AXIS, REC, STATS>(a, st);
    if (lim == LIM_TVD5) return launch_face_one<NV, 8, LIM_TVD5, AXIS, REC, STATS>(a, st);
    if constexpr (!REC)
      if (lim == LIM_VA) return launch_face_one<NV, 8, LIM_VA, AXIS, false, STATS>(a, st);
  }
  return cudaErrorNotSupported;
}

template <int NV, bool REC, bool STATS = false>
static cudaError_t launch_face_nv(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st) {
  static_assert(!(REC && STATS), "statistics kernels do not record");
  if (axis == 0) return launch_face_axis<NV, 0, REC, STATS>(a, K, lim, st);
  if constexpr (NV >= 4)
    if (axis == 1) return launch_face_axis<NV, 1, REC, STATS>(a, K, lim, st);
  if constexpr (NV >= 5)
    if (axis == 2) return launch_face_axis<NV, 2, REC, STATS>(a, K, lim, st);
  return cudaErrorNotSupported;
}

/* adjoint sweep with flags (or branches decided again) */
template <int NV, int K, int LIM, int AXIS>
static cudaError_t launch_adj_one(const AdjArgs& a, cudaStream_t st) {
  static AttrOnce attr;
  return launch_tile(adj_face_kernel<NV, K, LIM, AXIS>, attr, AdjTile<NV, K, AXIS>::SMEM, NV, AXIS, a.n, K, st,
                     &a);
}

/* adjoint sweep from a recorded linearisation (no limiter dependence) */
template <int NV, int K, int AXIS>
static cudaError_t launch_adj_lin_one(const AdjArgs& a, cudaStream_t st) {
  static AttrOnce attr;
  return launch_tile(adj_lin_kernel<NV, K, AXIS>, attr, AdjLinTile<NV, K, AXIS>::SMEM, NV, AXIS, a.n, K, st, &a);
}

template <int NV, int AXIS>
static cudaError_t launch_adj_axis(const AdjArgs& a, int K, int lim, cudaStream_t st) {
  if (a.lin) {
    if (K == 6) return launch_adj_lin_one<NV, 6, AXIS>(a, st);
    if (K == 8) return launch_adj_lin_one<NV, 8, AXIS>(a, st);
    return cudaErrorNotSupported;
  }
  if (K == 6) {
    if (lim == LIM_MP) return launch_adj_one<NV, 6, LIM_MP, AXIS>(a, st);
    if (lim == LIM_TVD5) return launch_adj_one<NV, 6, LIM_TVD5, AXIS>(a, st);
  } else if (K == 8) {
    if (lim == LIM_MP) return launch_adj_one<NV, 8, LIM_MP, AXIS>(a, st);
    if (lim == LIM_TVD5) return launch_adj_one<NV, 8, LIM_TVD5, AXIS>(a, st);
  }
  return cudaErrorNotSupported;
}

template <int NV>
static cudaError_t launch_adj_nv(const AdjArgs& a, int axis, int K, int lim, cudaStream_t st) {
  if (axis == 0) return launch_adj_axis<NV, 0>(a, K, lim, st);
  if constexpr (NV >= 4)
    if (axis == 1) return launch_adj_axis<NV, 1>(a, K, lim, st);
  if constexpr (NV >= 5)
    if (axis == 2) return launch_adj_axis<NV, 2>(a, K, lim, st);
  return cudaErrorNotSupported;
}

}  // namespace tenom
