// Instantiations of the several-M tile kernel (Section 3.4; fpw_tile.cuh).
#include "fpw_tile.cuh"

namespace fpw {

const void* tile_fn_multi(int R, int phase_mode) {
  const bool fp32p = phase_mode == FPW_PHASE_FP32;
#define FPW_INST(RR)                                                                      \
  if (R == RR)                                                                            \
    return fp32p ? (const void*)&tile_kernel_multi<RR, FPW_PHASE_FP32>                    \
                 : (const void*)&tile_kernel_multi<RR, FPW_PHASE_FIXED64>;
  FPW_INST(1)
  FPW_INST(2)
  FPW_INST(4)
  FPW_INST(8)
#undef FPW_INST
  return nullptr;
}

}  // namespace fpw
