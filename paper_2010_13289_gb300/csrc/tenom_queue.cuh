/* Warp work queue of the face kernels (tenom_face.cuh, tenom_face_fwd.cuh). */
#pragma once
#include "tenom_recon.cuh"

namespace tenom {

constexpr int QSLOTS = 64;     /* reconstruction queue items per warp: two sides x 32 lanes */

/* Warp work queue for the two reconstructions (f+, f-) of one characteristic field.
 * After the certified FP32 cutoff decisions, a side whose candidates are all smooth takes
 * the K-point central formula in its own lane; every other side (nonsmooth candidates, or
 * decisions the filter could not certify) is queued in shared memory and the warp's
 * active lanes work through the queue together, so the long general path (FP64 decisions,
 * candidates, limiter, assembly) runs with full lanes instead of once per side under
 * divergence.  wq: this warp's queue, QSLOTS items x (K + 2) doubles, component-major
 * (values, result, header); am: the warp's active lanes.  WT: the frozen linear weights
 * of each side (teno_general) come back in wp / wm. */
/* queue item r: the K stencil values and a header (decided flag bits, or undecided) */
template <int K>
__device__ __forceinline__ void queue_put(double* wq, int r, const double (&v)[K], bool decided, unsigned flag) {
#pragma unroll
  for (int q = 0; q < K; ++q) wq[q * QSLOTS + r] = v[q];
  wq[(K + 1) * QSLOTS + r] = __longlong_as_double(decided ? (0x100ll | flag) : 0ll);
}

/* the lanes in am work through queue items 0..n-1: FP64 decisions where undecided, then
   the general reconstruction; item r's result goes to slot K, its flag byte to slot K + 1 */
template <int K, int LIM>
__device__ __forceinline__ void queue_process(double* wq, int n, unsigned am, const SchemeDev& S, int& st) {
  const unsigned lt = (1u << (threadIdx.x & 31u)) - 1u;
  const int wl = __popc(am & lt), na = __popc(am);
  for (int base = 0; base < n; base += na) {
    const int it = base + wl;
    if (it < n) {
      double v[K];
#pragma unroll
      for (int q = 0; q < K; ++q) v[q] = wq[q * QSLOTS + it];
      const long long h = __double_as_longlong(wq[(K + 1) * QSLOTS + it]);
      unsigned bits = (unsigned)h & 63u;
      int ex = 7 + (int)((h >> 6) & 3);
      if (!(h & 0x100ll)) teno_decide_fp64<K>(v, S, bits, ex, st);
      wq[K * QSLOTS + it] = teno_general<K, LIM>(v, S, bits);
      wq[(K + 1) * QSLOTS + it] = __longlong_as_double((long long)(bits | ((unsigned)((ex - 7) & 3) << 6)));
    }
  }
}

}  // namespace tenom
