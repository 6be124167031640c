/* Internal declarations shared by the library's translation units. */
#pragma once
#include <cuda_runtime.h>
#include "tenom_face.cuh"

namespace tenom {

/* Launch the face kernel of (NV, K, limiter, axis); returns a CUDA error code. */
cudaError_t launch_face_nv3(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st);
cudaError_t launch_face_nv4(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st);
cudaError_t launch_face_nv5(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st);
/* The same, also writing the face linearisation to a.lin (record kernels). */
cudaError_t launch_face_rec_nv3(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st);
cudaError_t launch_face_rec_nv4(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st);
cudaError_t launch_face_rec_nv5(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st);
/* The face kernel's decision statistics (tenom_stats.cuh) added to a.stats; no fluxes. */
cudaError_t launch_stats_nv3(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st);
cudaError_t launch_stats_nv4(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st);
cudaError_t launch_stats_nv5(const FaceArgs& a, int axis, int K, int lim, cudaStream_t st);

/* Launch geometry of a face sweep (kept in one place for the tests of the host logic):
   tiles over the n_a + 1 faces of a line, or over n_a faces (wrapped: a forward kernel on
   a periodic axis, whose face n_a is face 0's copy); fwd_tile: the forward and record
   kernels' tiles (fx_faces(K, nv) along x; FWD_LANES x columns in y/z), else FX_FACES along x
   and 32 x columns x ft_faces(K). */
inline void face_grid(int nv, int axis, const int* n, int K, dim3* grid, dim3* block, bool wrapped = false,
                      bool fwd_tile = false) {
  const int nf = n[axis] + (wrapped ? 0 : 1);
  if (axis == 0) {
    const int fx = fwd_tile ? fx_faces(K, nv) : FX_FACES;
    *block = dim3(fx);
    *grid = dim3((unsigned)(n[1] * n[2]), (unsigned)((nf + fx - 1) / fx));
  } else {
    const int other = (axis == 1) ? n[2] : n[1];
    const int lanes = fwd_tile ? FWD_LANES : 32;
    const int ft = fwd_tile ? fx_faces(K, nv) / FWD_LANES : ft_faces(K);
    *block = dim3(lanes * ft);
    *grid = dim3((unsigned)((n[0] + lanes - 1) / lanes), (unsigned)((nf + ft - 1) / ft), (unsigned)other);
  }
}

}  // namespace tenom

#include <string>
#include "tenom.h"

namespace tenom {
/* Argument checks of tenom_create, usable without a context. */
tenom_status check_grid_scheme(const tenom_grid* g, const tenom_scheme* s, std::string* msg);
/* Device copy of a scheme (all-zero d_k replaced by the maximal-order weights). */
SchemeDev scheme_for_device(const tenom_scheme& s);
/* dUdt = -sum_a (F_a[f+1] - F_a[f]) / dx_a from face buffers F[a] ([nv][nface_a]). */
cudaError_t launch_rhs_divergence(int nv, double* const F[3], const int n[3], const double dx[3], long long ncell,
                                  const long long nface[3], double* out, cudaStream_t st);
}  // namespace tenom

namespace tenom {
struct AdjArgs;
/* Launch the adjoint face sweep of (NV, K, limiter, axis): Z += L_a'(U)^T w, from a.lin (the
   recorded linearisation) when set, else from a.flags (or branches decided again). */
cudaError_t launch_adj_nv3(const AdjArgs& a, int axis, int K, int lim, cudaStream_t st);
cudaError_t launch_adj_nv4(const AdjArgs& a, int axis, int K, int lim, cudaStream_t st);
cudaError_t launch_adj_nv5(const AdjArgs& a, int axis, int K, int lim, cudaStream_t st);
}  // namespace tenom
