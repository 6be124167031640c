/* Recording face-kernel instantiations for nvar = 3 (1D Euler): the forward face flux
 * plus its frozen-branch linearisation. */
#include "tenom_launch.cuh"

namespace tenom {

cudaError_t launch_face_rec_nv3(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st) {
  return launch_face_nv<3, true>(a, axis, K, lim, st);
}

}  // namespace tenom
