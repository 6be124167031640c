/* Decision-statistics face-kernel instantiations for nvar = 5 (3D Euler): the face
 * kernel's characteristic sequences, counted instead of reconstructed (tenom_stats.cuh). */
#include "tenom_launch.cuh"

namespace tenom {

cudaError_t launch_stats_nv5(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st) {
  return launch_face_nv<5, false, true>(a, axis, K, lim, st);
}

}  // namespace tenom
