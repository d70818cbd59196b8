// Host side of the persistent FPW tile kernels (device templates in
// fpw_tile.cuh): shared-memory sizes, kernel selection and launches, and the
// per-tile grid-deviation kernel that decides which tiles may step the phase
// linearly (Appendix A.1 bins on a linear grid, Section 4's frequency sweep).
#include <math.h>

#include "fpw_tile.cuh"

namespace fpw {
namespace {

__device__ __forceinline__ double dev_warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Per tile q (start s = q*Wown - 1, width W = Wown + 2): the largest deviation
// of the grid from the line through f_a (a = max(s, 0)) with step df, the
// linear prediction used by the tile kernel's fixed-point stepping.
__global__ void tile_dev_kernel(const double* freqs, int64_t F, int W, int64_t tiles, double* dev) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const double df = (F > 1) ? (freqs[F - 1] - freqs[0]) / (double)(F - 1) : 0.0;
  for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < tiles; q += warps) {
    const int64_t s = q * (W - 2) - 1;
    const int64_t a = s < 0 ? 0 : s;
    const double fa = freqs[a];
    double d = 0.0;
    for (int j = lane; j < W; j += 32) {
      const int64_t k = s + j;
      if (k >= 0 && k < F) d = fmax(d, fabs(freqs[k] - fma((double)(k - a), df, fa)));
    }
    d = dev_warp_max(d);
    if (lane == 0) dev[q] = d;
  }
}

const void* pick(int R, int phase_mode, int accum, bool multi, bool dump, int spec = 0) {
  if (multi) return dump ? nullptr : tile_fn_multi(R, phase_mode, spec);
  switch (accum) {
    case FPW_ACCUM_FP32:
      return (R == 3 || R == 5 || R == 6) ? tile_fn_f32_odd(R, phase_mode, dump) : tile_fn_f32(R, phase_mode, dump);
    case FPW_ACCUM_FP64: return tile_fn_f64(R, phase_mode, dump);
    case FPW_ACCUM_FP32_COMP: return tile_fn_comp(R, phase_mode, dump);
    default: return nullptr;
  }
}

}  // namespace

size_t tile_smem_bytes(int T, int R, int M, int NC, int /*k*/, int accum, int ngroups) {
  return tile_layout(T, R, M, NC, accum_bin_bytes(accum), ngroups).total;
}

bool tile_supported_R(int R) { return R >= 1 && R <= 8 && R != 7; }

bool tile_has_R(int R, int accum, bool multi) {
  if (R == 1 || R == 2 || R == 4 || R == 8) return true;
  return (R == 3 || R == 5 || R == 6) && accum == FPW_ACCUM_FP32 && !multi;
}

cudaError_t tile_init_attributes(int max_smem) {
  for (int R : {3, 5, 6})
    for (int ph : {FPW_PHASE_FIXED64, FPW_PHASE_FP32})
      for (bool dump : {false, true}) {
        cudaError_t e =
            cudaFuncSetAttribute(pick(R, ph, FPW_ACCUM_FP32, false, dump), cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
      }
  for (int R : {1, 2, 4, 8})
    for (int ph : {FPW_PHASE_FIXED64, FPW_PHASE_FP32}) {
      for (int acc : {FPW_ACCUM_FP32, FPW_ACCUM_FP64, FPW_ACCUM_FP32_COMP})
        for (bool dump : {false, true}) {
          cudaError_t e =
              cudaFuncSetAttribute(pick(R, ph, acc, false, dump), cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
          if (e != cudaSuccess) return e;
        }
      for (int spec = 0; spec <= 3; ++spec) {  // the generic kernel where no compiled one exists
        cudaError_t e = cudaFuncSetAttribute(pick(R, ph, FPW_ACCUM_FP32, true, false, spec),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
      }
    }
  return cudaSuccess;
}

int tile_max_blocks_per_sm(int R, int phase_mode, int accum, int T, size_t smem, bool multi, bool dump, int spec) {
  const void* fn = pick(R, phase_mode, accum, multi, dump, spec);
  if (!fn) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, T, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_tile_dev(const double* freqs, int64_t F, int W, int64_t tiles, double* dev, cudaStream_t st) {
  if (tiles <= 0) return cudaSuccess;
  int64_t blocks = (tiles + 7) / 8;
  blocks = blocks > 4096 ? 4096 : blocks;
  tile_dev_kernel<<<(unsigned)blocks, 256, 0, st>>>(freqs, F, W, tiles, dev);
  return cudaGetLastError();
}

cudaError_t launch_tile(const TileArgs& a, const TileShape& s, int phase_mode, int accum, int grid, cudaStream_t st) {
  const void* fn = pick(s.R, phase_mode, accum, a.ngroups > 0, a.bins_out != nullptr,
                        multi_spec_of(a.M, a.ngroups, a.group_g));
  if (!fn) return cudaErrorInvalidValue;
  void* params[] = {const_cast<TileArgs*>(&a)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(s.threads), params, s.smem, st);
}

}  // namespace fpw
