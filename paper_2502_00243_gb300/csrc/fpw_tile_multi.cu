// Instantiations of the several-M tile kernel (Section 3.4; fpw_tile.cuh): the
// generic combination for every R and phase mode, and the compiled
// combinations (multi_spec_of) at the frequencies per thread their bin counts
// take by default (M_max = 60: R = 1, 40: R = 2, 20: R = 4) with the fixed64
// phase. Other (R, phase) pairs of a compiled spec run the generic kernel.
#include "fpw_tile.cuh"

namespace fpw {

const void* tile_fn_multi(int R, int phase_mode, int spec) {
  const bool fp32p = phase_mode == FPW_PHASE_FP32;
  if (!fp32p) {
    if (spec == 1 && R == 1) return (const void*)&tile_kernel_multi<1, FPW_PHASE_FIXED64, 1>;
    if (spec == 2 && R == 2) return (const void*)&tile_kernel_multi<2, FPW_PHASE_FIXED64, 2>;
    if (spec == 3 && R == 4) return (const void*)&tile_kernel_multi<4, FPW_PHASE_FIXED64, 3>;
  }
#define FPW_INST(RR)                                                                      \
  if (R == RR)                                                                            \
    return fp32p ? (const void*)&tile_kernel_multi<RR, FPW_PHASE_FP32, 0>                 \
                 : (const void*)&tile_kernel_multi<RR, FPW_PHASE_FIXED64, 0>;
  FPW_INST(1)
  FPW_INST(2)
  FPW_INST(4)
  FPW_INST(8)
#undef FPW_INST
  return nullptr;
}

}  // namespace fpw
