/* Batched stage kernels with the positivity-preserving flux limiter (Section 4.4), in a
   translation unit of their own so that they compile in parallel with the others. */
#include "tenom_batch_kernel.cuh"

namespace tenom {

template <int K, int LIM, int TILE>
static StageFn stage_fn_pp() { return batch_stage_kernel<K, LIM, TILE, true>; }

StageFn pick_stage_pp(int K, int lim, int tile) {
#define TENOM_PICK(KK, LL, TT) if (K == KK && lim == LL && tile == TT) return stage_fn_pp<KK, LL, TT>();
  TENOM_PICK(6, LIM_MP, 64) TENOM_PICK(6, LIM_MP, 128) TENOM_PICK(6, LIM_MP, 256)
  TENOM_PICK(6, LIM_TVD5, 64) TENOM_PICK(6, LIM_TVD5, 128) TENOM_PICK(6, LIM_TVD5, 256)
  TENOM_PICK(8, LIM_MP, 64) TENOM_PICK(8, LIM_MP, 128) TENOM_PICK(8, LIM_MP, 256)
  TENOM_PICK(8, LIM_TVD5, 64) TENOM_PICK(8, LIM_TVD5, 128) TENOM_PICK(8, LIM_TVD5, 256)
#undef TENOM_PICK
  return nullptr;
}

}  // namespace tenom
