// Declarations of the shared-timestamp path (fpw_shared.cu): curves observed
// at the same times, binned together on the tensor cores.
#pragma once
#include "fpw_internal.cuh"

namespace fpw {

// Curves sharing one set of observation times (fpw_shared.cu).
struct SharedArgs {
  const double* t;          // [n] shared times
  int64_t n;
  int64_t ncurves;
  const double* x;          // [ncurves][n]
  const double* sigma;      // [ncurves][n]
  const double* freqs;      // [nfreq]
  int64_t nfreq;
  int M;
  int fpm;                  // frequencies per accumulator (256 / M)
  int n_mma;                // MMA N: fpm * M rounded up to 16
  int64_t npass;            // frequency passes of 2 * fpm frequencies
  int64_t ngroups;          // groups of 64 curves
  int64_t nchunks;          // chunks of 32 observations
  unsigned char* image;     // fp16 hi/lo operand image [ngroups][nchunks][16 KB]
  float* inv_scale;         // [ngroups * 64][2]: 2^-e for a and w
  unsigned long long* step; // [n] 64-bit phase step frac(t_i df) of the grid's mean spacing df
  unsigned long long* tmax_bits;  // max |t| (binary64 bits)
  uint8_t* curve_bad;       // [ngroups * 64]
  unsigned* status;
  double inv_alpha2;
  float* S32;               // dense [ncurves][nfreq] FP32 (required when k > 0), or NULL
  double* S_out;            // dense [ncurves][nfreq] or NULL
  float* scratch32;         // [32 * 64] write sink for padding curves
  double* scratch64;        // [32 * 64]
  int k;
  int peak_raw;
  int32_t* topk_idx;        // [ncurves][k]
  float* topk_S;
  cudaEvent_t timing_start; // optional events around the MMA kernel
  cudaEvent_t timing_stop;
};

size_t shared_image_bytes(int64_t ncurves, int64_t n);
int shared_curves_per_group();
int shared_freqs_per_mma(int M, int* n_mma);  // 0 if M is unsupported
size_t shared_smem_bytes();
cudaError_t shared_init_attributes();
cudaError_t launch_shared(const SharedArgs& a, int nsm, cudaStream_t st);

}  // namespace fpw
