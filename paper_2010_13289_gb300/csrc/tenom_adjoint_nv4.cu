/* Adjoint face-kernel instantiations for nvar = 4 (flags and linearisation-tape sweeps). */
#include "tenom_launch.cuh"

namespace tenom {

cudaError_t launch_adj_nv4(const AdjArgs& a, int axis, int K, int lim, cudaStream_t st) {
  return launch_adj_nv<4>(a, axis, K, lim, st);
}

}  // namespace tenom
