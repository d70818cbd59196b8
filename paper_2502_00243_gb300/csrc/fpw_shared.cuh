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
  long long wait_clocks;    // limit of each pipeline wait in SM clocks (0: the default, about 2 s)
};

// Per-curve top-k peaks of a dense FP32 periodogram [ncurves][nfreq] (one block per curve).
struct DenseTopk32Args {
  const float* S32;
  int64_t nfreq;
  int k;
  int peak_raw;
  const uint8_t* curve_bad;  // [ncurves]: no peaks for a bad curve
  const unsigned* status;    // kStatusGrid: no peaks at all
  int32_t* topk_idx;         // [ncurves][k]
  float* topk_S;
};
cudaError_t launch_dense_topk32(const DenseTopk32Args& t, int64_t ncurves, cudaStream_t st);

// Baseline-drift statistic for a ragged batch (fpw_drift.cu).
struct DriftArgs {
  const int64_t* offsets;   // [ncurves + 1]
  int64_t ncurves;
  const double* t;
  const double* x;
  const double* sigma;
  const double* freqs;
  int64_t nfreq;
  int M;
  int K;                    // Chebyshev basis functions (0..4)
  double beta;              // prior standard deviation of each basis coefficient
  double inv_alpha2;
  void* payload;            // [nobs] 32-byte per-observation records (prep kernel)
  double* tabs;             // [ncurves] max |t| of the curve's finite times
  double* H0;               // [ncurves][4][4]: I + B^T D B
  double* g;                // [ncurves][4]: H0^-1 B^T D x
  uint8_t* curve_bad;       // [ncurves]
  unsigned* status;
  float* S32;               // dense [ncurves][nfreq] (required when k > 0), or NULL
  double* S_out;            // dense [ncurves][nfreq] or NULL
  int k;
  int peak_raw;
  int32_t* topk_idx;
  float* topk_S;
  cudaEvent_t timing_start;
  cudaEvent_t timing_stop;
};
int drift_threads(int M, int K, int smem_optin);  // threads per block, 0 if M is too large
size_t drift_smem_bytes(int M, int K, int T, int R);  // R frequencies per thread (1 or 2)
bool drift_fits(int M, int K, int T, int R, int smem_optin);
int drift_max_basis();
size_t drift_payload_bytes();
cudaError_t drift_init_attributes(int max_smem);
cudaError_t launch_drift(const DriftArgs& a, int T, int R, cudaStream_t st);

size_t shared_image_bytes(int64_t ncurves, int64_t n);
int shared_curves_per_group();
int shared_freqs_per_mma(int M, int* n_mma);  // 0 if M is unsupported
size_t shared_smem_bytes();
cudaError_t shared_init_attributes();
cudaError_t launch_shared(const SharedArgs& a, int nsm, cudaStream_t st);

}  // namespace fpw
