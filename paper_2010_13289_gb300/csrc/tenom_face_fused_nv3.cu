/* Instantiations for nvar = 3 (1D Euler) of the x sweep with the cell update fused (flux
 * difference and SSP-RK3 stage combine in the tile, see face_kernel). */
#include "tenom_launch.cuh"

namespace tenom {

cudaError_t launch_fused_nv3(const FaceArgs& a, int K, int lim, cudaStream_t st) {
  return launch_fused_nv<3>(a, K, lim, st);
}

}  // namespace tenom
