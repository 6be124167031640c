/* Adjoint face-kernel instantiations for nvar = 4. */
#include "tenom_internal.h"
#include "tenom_adjoint_kernels.cuh"

namespace tenom {

template <int NV, int K, int LIM, int AXIS>
static cudaError_t launch_adj_one(const AdjArgs& a, cudaStream_t st) {
  using T = AdjTile<NV, K, AXIS>;
  auto kern = adj_face_kernel<NV, K, LIM, AXIS>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  dim3 grid, block;
  face_grid(NV, AXIS, a.n, K, &grid, &block);
  kern<<<grid, block, T::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <int NV, int AXIS>
static cudaError_t launch_adj_axis(const AdjArgs& a, int K, int lim, cudaStream_t st) {
  if (K == 6) {
    if (lim == LIM_MP) return launch_adj_one<NV, 6, LIM_MP, AXIS>(a, st);
    if (lim == LIM_TVD5) return launch_adj_one<NV, 6, LIM_TVD5, AXIS>(a, st);
  } else if (K == 8) {
    if (lim == LIM_MP) return launch_adj_one<NV, 8, LIM_MP, AXIS>(a, st);
    if (lim == LIM_TVD5) return launch_adj_one<NV, 8, LIM_TVD5, AXIS>(a, st);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_adj_nv4(const AdjArgs& a, int axis, int K, int lim, cudaStream_t st) {
  if (axis == 0) return launch_adj_axis<4, 0>(a, K, lim, st);
  if (axis == 1) return launch_adj_axis<4, 1>(a, K, lim, st);
  return cudaErrorNotSupported;
}

}  // namespace tenom
