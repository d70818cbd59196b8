// Instantiations of the tile kernel with binary64 bin sums (fpw_tile.cuh).
#include "fpw_tile.cuh"

namespace fpw {

const void* tile_fn_f64(int R, int phase_mode, bool dump) {
  const bool fp32p = phase_mode == FPW_PHASE_FP32;
#define FPW_INST(RR)                                                                                         \
  if (R == RR) {                                                                                             \
    if (dump)                                                                                                \
      return fp32p ? (const void*)&tile_kernel<RR, FPW_PHASE_FP32, AccF64, true>                                 \
                   : (const void*)&tile_kernel<RR, FPW_PHASE_FIXED64, AccF64, true>;                             \
    return fp32p ? (const void*)&tile_kernel<RR, FPW_PHASE_FP32, AccF64, false>                                  \
                 : (const void*)&tile_kernel<RR, FPW_PHASE_FIXED64, AccF64, false>;                              \
  }
  FPW_INST(1)
  FPW_INST(2)
  FPW_INST(4)
  FPW_INST(8)
#undef FPW_INST
  return nullptr;
}

}  // namespace fpw
