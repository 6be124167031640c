/* Forward face-kernel instantiations for nvar = 3 (1D Euler). */
#include "tenom_launch.cuh"

namespace tenom {

cudaError_t launch_face_nv3(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st) {
  return launch_face_nv<3, false>(a, axis, K, lim, st);
}

}  // namespace tenom
