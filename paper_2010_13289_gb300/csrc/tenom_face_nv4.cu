/* Forward face-kernel instantiations for nvar = 4 (2D Euler). */
#include "tenom_launch.cuh"

namespace tenom {

cudaError_t launch_face_nv4(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st) {
  return launch_face_nv<4, false>(a, axis, K, lim, st);
}

}  // namespace tenom
