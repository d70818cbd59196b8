// Internal declarations of the GB300 FPW library: kernel argument blocks,
// device-side phase arithmetic and launch wrappers. Not part of the public ABI
// (include/fpw.h is).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fpw.h"

namespace fpw {

// Device status bits latched in the context's status word.
constexpr unsigned kStatusData = 1u;     // sigma <= 0 or non-finite t/x/sigma in some curve
constexpr unsigned kStatusGrid = 2u;     // non-finite frequency
constexpr unsigned kStatusTimeout = 4u;  // a bounded wait gave up

// Largest distance (cycles) by which the linear-grid fast path may move a
// phase relative to frac(t_i * freqs[k]): tiles whose grid deviates more are
// evaluated with a direct per-frequency anchor instead.
constexpr double kGridTolCycles = 2e-10;

// Largest number of derived bin counts computed from one M_max pass.
constexpr int kMaxGroups = 8;

// Several-M calls whose (M_max, groups) have a compiled combination in the
// tile kernel (1: M_max = 60 with groups 3, 6, 15; 2: 40 with 2, 4, 10; 3: 20
// with 1, 2, 4; groups in that order), else 0 (the generic combination).
inline int multi_spec_of(int M, int ngroups, const int* g) {
  if (ngroups != 3) return 0;
  if (M == 60 && g[0] == 3 && g[1] == 6 && g[2] == 15) return 1;
  if (M == 40 && g[0] == 2 && g[1] == 4 && g[2] == 10) return 2;
  if (M == 20 && g[0] == 1 && g[1] == 2 && g[2] == 4) return 3;
  return 0;
}

// One unit of persistent work: frequencies [f_lo, f_hi) of curve `curve`.
// Its top-k candidates go to row `slot` of the candidate table.
struct WorkItem {
  int32_t curve;
  int32_t f_lo;
  int32_t f_hi;
  int32_t slot;
};

struct TileArgs {
  const double* t;           // observation times, CSR by curve
  const int64_t* offsets;    // [ncurves + 1]; NULL: one curve of n_single observations
  int64_t n_single;
  const void* aw;            // prep output per observation: float2 {a = x w, w = 1/sigma^2}, double2, or
                             // float4 {a_hi, w_hi, a_lo, w_lo} (compensated sums)
  const double* freqs;       // [nfreq]
  int64_t nfreq;
  const WorkItem* items;     // [nitems], cost-descending
  int nitems;
  unsigned* counter;         // work-queue head (zeroed before launch)
  unsigned* status;          // latched status bits
  const uint8_t* curve_bad;  // [ncurves] 1 = invalid data
  double* cand_S;            // [slots * k] candidate peaks (S), or NULL when k == 0
  int32_t* cand_idx;         // [slots * k]
  double* S_out;             // dense [ncurves * nfreq] or NULL
  int M;
  int k;
  int peak_raw;
  int K;                     // FPW_PHASE_FP32 re-anchor interval
  int obs_chunk;             // observations staged per pass
  double inv_alpha2;
  const double* tile_dev;    // per-tile grid deviation (tile_dev_kernel), or NULL: checked in the tile kernel
  int ngroups;               // several-M kernel: number of groups (0 = the single-M kernel)
  int group_g[kMaxGroups];   // M = M / group_g[q] for group q
  int64_t group_rows;        // candidate rows per group (cand tables are [group][slot][k])
  int32_t* bins_out;         // NULL, or bins of (k, i) for bins_k0 <= k < bins_k1 at [(k - bins_k0) * bins_nobs + i]
  int64_t bins_k0, bins_k1, bins_nobs;
};

struct PrepArgs {
  const double* t;
  const double* x;
  const double* sigma;
  const int64_t* offsets;  // NULL: one curve
  int64_t ncurves;
  int64_t nobs;
  const double* freqs;
  int64_t nfreq;
  void* aw;                // [nobs] float2, double2 or float4 (see TileArgs::aw), or NULL
  int accum;               // FPW_ACCUM_*
  uint8_t* curve_bad;      // [ncurves], zeroed before launch
  unsigned* status;
};

struct MergeArgs {
  const double* cand_S;
  const int32_t* cand_idx;
  const int32_t* cand_base;  // [ncurves + 1] candidate rows per curve
  const uint8_t* curve_bad;
  const unsigned* status;
  int64_t ncurves;
  int k;
  int32_t* topk_idx;         // curve c's list starts at c * out_stride (out_stride = k when 0)
  float* topk_S;
  int out_stride;
  int32_t* topk_off;         // several-M: receives key & 63 (the bin offset); topk_idx then gets key >> 6
  int max_rows;              // most candidate rows of one curve (0: unknown); many rows take a block per curve
};

struct PlainArgs {           // binary64 plain form, one curve
  const double* t;
  const double* x;
  const double* sigma;
  int64_t n;
  const double* freqs;
  int64_t nfreq;
  int M;
  double inv_alpha2;
  double* S_out;             // [nfreq]
  unsigned* status;
  int32_t* bins_out;         // NULL, or bins of (k, i) for bins_k0 <= k < bins_k1 at
  int64_t bins_k0, bins_k1;  //   [(k - bins_k0) * bins_nobs + bins_base + i]
  int64_t bins_nobs, bins_base;
};

struct DenseTopkArgs {       // top-k of one dense periodogram (plain form)
  const double* S;
  int64_t nfreq;
  int k;
  int peak_raw;
  int32_t* topk_idx;
  float* topk_S;
  const unsigned* status;
};

// Bytes of one tile-kernel bin (A, B [, cA, cB]) and of one staged weight
// record per accumulation mode (FPW_ACCUM_*).
__host__ __device__ constexpr size_t accum_bin_bytes(int accum) { return accum == FPW_ACCUM_FP32 ? 8 : 16; }

// Tile-kernel shape chosen by the host (tuned per bin count and curve size).
struct TileShape {
  int threads;   // T
  int R;         // frequencies per thread
  int obs_chunk; // NC
  size_t smem;   // dynamic shared memory bytes
  int items;     // work items per resident block in the persistent schedule
};

// ---- launch wrappers (defined in the .cu files) -------------------------
size_t tile_smem_bytes(int T, int R, int M, int NC, int k, int accum, int ngroups = 0);
int tile_max_blocks_per_sm(int R, int phase_mode, int accum, int T, size_t smem, bool multi = false,
                           bool dump = false, int spec = 0);  // spec: the several-M combination (fpw_tile.cuh)
bool tile_supported_R(int R);                      // some tile kernel has R frequencies per thread
bool tile_has_R(int R, int accum, bool multi);     // the kernel for this sum mode / several-M call has it
// Launches the kernel for (R, phase, accum); several-M when a.ngroups > 0, the
// bin-dumping instantiation when a.bins_out != NULL.
cudaError_t launch_tile(const TileArgs& a, const TileShape& s, int phase_mode, int accum, int grid, cudaStream_t st);
cudaError_t launch_prep(const PrepArgs& a, cudaStream_t st);
// Per-tile grid deviation for tiles of width W starting at q*(W-2)-1, q < tiles.
cudaError_t launch_tile_dev(const double* freqs, int64_t F, int W, int64_t tiles, double* dev, cudaStream_t st);
cudaError_t launch_merge(const MergeArgs& a, cudaStream_t st);
cudaError_t launch_plain(const PlainArgs& a, cudaStream_t st);
cudaError_t launch_dense_topk(const DenseTopkArgs& a, cudaStream_t st);
cudaError_t launch_latch(unsigned* words, cudaStream_t st);  // words[2] |= words[1]
cudaError_t launch_fill_topk(int32_t* idx, float* S, int64_t n, cudaStream_t st);
cudaError_t tile_init_attributes(int max_smem);
cudaError_t plain_init_attributes(int max_smem);
size_t plain_smem_bytes(int M);
cudaError_t launch_entropy_dense(const double* t, int64_t n, const double* freqs, int64_t nfreq, int M, float* H_out,
                                 cudaStream_t st);
cudaError_t launch_entropy_peaks(const int64_t* offsets, int64_t ncurves, const double* t, const double* freqs,
                                 int64_t nfreq, int M, int k, const int32_t* topk_idx, float* H_out, float* z_out,
                                 cudaStream_t st);

// ---- device arithmetic --------------------------------------------------
#ifdef __CUDACC__

// v = mant * 2^e2 exactly (mant < 2^53); sign dropped.
__device__ __forceinline__ void split_binary64(double v, unsigned long long& mant, int& e2) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7ffull);
  mant = b & 0xFFFFFFFFFFFFFull;
  if (be == 0) {
    e2 = -1074;  // zero or subnormal
  } else {
    mant |= 1ull << 52;
    e2 = be - 1075;
  }
}

// Phase of t*f as a 64-bit fixed-point fraction of a cycle, rounded UP:
//   returns ceil(frac(t*f) * 2^64) (mod 2^64),
// computed exactly from the integer product of the two binary64 significands
// (no binary64 arithmetic: the 106-bit product is formed with integer
// multiplies and the 64 bits just below the binary point are extracted).
// Rounding up makes every anchor and step an upper bound of the exact value,
// so a phase stepped from them never falls below the exact phase: a phase
// exactly on a bin edge stays in the upper bin (bins are half-open), as in
// exact arithmetic. For t*f < 0 the result is -floor(frac(|t f|) 2^64) mod 2^64,
// also an upper bound. t and f must be finite.
__device__ __forceinline__ unsigned long long phase_fixed64(double t, double f) {
  unsigned long long mt, mf;
  int et, ef;
  split_binary64(t, mt, et);
  split_binary64(f, mf, ef);
  const unsigned long long lo = mt * mf;
  const unsigned long long hi = __umul64hi(mt, mf);
  const int s = et + ef + 64;  // frac * 2^64 = (Q * 2^s) mod 2^64, Q = hi * 2^64 + lo
  unsigned long long r;
  bool inexact;
  if (s >= 64) {
    r = 0ull;
    inexact = false;
  } else if (s >= 0) {
    r = lo << s;
    inexact = false;
  } else {
    const int sh = -s;
    if (sh < 64) {
      r = (lo >> sh) | (hi << (64 - sh));
      inexact = (lo << (64 - sh)) != 0ull;
    } else if (sh < 128) {
      r = hi >> (sh - 64);
      inexact = lo != 0ull || (sh > 64 && (hi << (128 - sh)) != 0ull);
    } else {
      r = 0ull;
      inexact = (lo | hi) != 0ull;
    }
  }
  const bool neg = ((__double_as_longlong(t) ^ __double_as_longlong(f)) < 0) && (mt != 0ull) && (mf != 0ull);
  return neg ? (0ull - r) : (r + (inexact ? 1ull : 0ull));
}

// Bin of a 64-bit fixed-point phase: floor(M * Phi_hi / 2^32). It equals
// floor(M * Phi / 2^64) except within 2^-32 cycles below a bin edge.
__device__ __forceinline__ unsigned bin_of_phase(unsigned long long phi, unsigned M) {
  return __umulhi((unsigned)(phi >> 32), M);
}

// Packed FP32 pair add (one f32x2 instruction on sm_100 and later).
__device__ __forceinline__ float2 f2add(float2 a, float2 b) {
  unsigned long long x, y, z;
  asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(z));
  return r;
}

// Ranking used for peaks: larger S first, then lower frequency index.
__device__ __forceinline__ bool ranks_before(double s1, int k1, double s2, int k2) {
  return (s1 > s2) || (s1 == s2 && (unsigned)k1 < (unsigned)k2);
}

#endif  // __CUDACC__

}  // namespace fpw
