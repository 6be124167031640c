/* Forward face-kernel instantiations for nvar = 5 (3D Euler). */
#include "tenom_launch.cuh"

namespace tenom {

cudaError_t launch_face_nv5(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st) {
  return launch_face_nv<5, false>(a, axis, K, lim, st);
}

}  // namespace tenom
