// Instantiations of the tile kernel with FP32 bin sums at R = 3, 5 and 6
// frequencies per thread (fpw_tile.cuh), for one M per call. With 128 threads
// they keep about 80-100 bin pairs per thread, two blocks per SM, at M = 26..33
// (R = 3), 17..20 (R = 5) and 13..16 (R = 6), where the neighbouring powers of
// two would leave the per-observation broadcast less amortised or fewer warps
// per SM. A separate translation unit so that it compiles in parallel with the
// others.
#include "fpw_tile.cuh"

namespace fpw {

const void* tile_fn_f32_odd(int R, int phase_mode, bool dump) {
  const bool fp32p = phase_mode == FPW_PHASE_FP32;
#define FPW_INST(RR)                                                                                         \
  if (R == RR) {                                                                                             \
    if (dump)                                                                                                \
      return fp32p ? (const void*)&tile_kernel<RR, FPW_PHASE_FP32, AccF32, true>                                 \
                   : (const void*)&tile_kernel<RR, FPW_PHASE_FIXED64, AccF32, true>;                             \
    return fp32p ? (const void*)&tile_kernel<RR, FPW_PHASE_FP32, AccF32, false>                                  \
                 : (const void*)&tile_kernel<RR, FPW_PHASE_FIXED64, AccF32, false>;                              \
  }
  FPW_INST(3)
  FPW_INST(5)
  FPW_INST(6)
#undef FPW_INST
  return nullptr;
}

}  // namespace fpw
