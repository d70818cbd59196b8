// Phase entropy of the observation times (Appendix C):
//   H(f) = -sum_m (N_m / N) log(N_m / N),  N_m observations in phase bin m,
// with Hutcheson's expectation and variance for equally likely bins,
//   E(H)   = log M - (M - 1) / (2 N) - (M - 1)(M + 1) / (12 N^2),
//   Var(H) = (M - 1) / (2 N^2) + (M^2 - 1) / (6 N^3),
// used to flag periodogram peaks whose phase coverage is anomalously uneven
// (z = (H - E) / sqrt(Var) strongly negative).
//
// Bins use the exact anchor of the periodogram kernels
// (bin_of_phase(phase_fixed64(t, f))), so they agree with the tile kernels'
// bins except within 2^-32 cycles of an edge.
#include <math.h>

#include "fpw_internal.cuh"

namespace fpw {
namespace {

constexpr int kEntThreads = 128;
constexpr int kEntChunk = 512;

// H from bin counts: log N - (1/N) sum_m N_m log N_m, in FP32 (the count
// terms are exact integers; the logarithms carry the rounding).
__device__ __forceinline__ float entropy_from_counts_sum(float sum_clogc, float N) {
  return N > 0.f ? logf(N) - sum_clogc / N : 0.f;
}

// One thread per frequency; observation times staged in shared memory; counts
// per (bin, thread) as 32-bit integers, [m][thread] (conflict-free).
__global__ void __launch_bounds__(kEntThreads) entropy_dense_kernel(const double* t, int64_t n, const double* freqs,
                                                                    int64_t nfreq, int M, float* H_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* st = reinterpret_cast<double*>(smem);
  unsigned* cnt = reinterpret_cast<unsigned*>(st + kEntChunk);
  const int tid = threadIdx.x;
  const int64_t k = (int64_t)blockIdx.x * kEntThreads + tid;
  const double f = freqs[k < nfreq ? k : nfreq - 1];
  for (int m = 0; m < M; ++m) cnt[m * kEntThreads + tid] = 0u;
  for (int64_t o = 0; o < n; o += kEntChunk) {
    const int c = (int)((n - o) < kEntChunk ? (n - o) : kEntChunk);
    __syncthreads();
    for (int i = tid; i < c; i += kEntThreads) st[i] = t[o + i];
    __syncthreads();
    for (int i = 0; i < c; ++i) {
      const unsigned m = bin_of_phase(phase_fixed64(st[i], f), (unsigned)M);
      cnt[m * kEntThreads + tid] += 1u;
    }
  }
  if (k < nfreq) {
    float s = 0.f;
    for (int m = 0; m < M; ++m) {
      const unsigned c = cnt[m * kEntThreads + tid];
      if (c > 1u) s += (float)c * logf((float)c);
    }
    H_out[k] = entropy_from_counts_sum(s, (float)n);
  }
}

// One warp per (curve, peak): counts in shared memory, H, then the z-score.
constexpr int kPeakWarps = 4;

__global__ void __launch_bounds__(kPeakWarps * 32) entropy_peaks_kernel(const int64_t* offsets, int64_t ncurves,
                                                                        const double* t, const double* freqs,
                                                                        int64_t nfreq, int M, int k,
                                                                        const int32_t* topk_idx, float* H_out,
                                                                        float* z_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned* cnt = reinterpret_cast<unsigned*>(smem) + warp * M;
  const int64_t total = ncurves * k;
  for (int64_t e = (int64_t)blockIdx.x * kPeakWarps + warp; e < total; e += (int64_t)gridDim.x * kPeakWarps) {
    const int64_t c = e / k;
    const int32_t fi = topk_idx[e];
    if (fi < 0 || fi >= nfreq) {
      if (lane == 0) {
        H_out[e] = __int_as_float(0x7fc00000);
        z_out[e] = __int_as_float(0x7fc00000);
      }
      continue;
    }
    for (int m = lane; m < M; m += 32) cnt[m] = 0u;
    __syncwarp();
    const double f = freqs[fi];
    const int64_t o0 = offsets[c], n = offsets[c + 1] - o0;
    for (int64_t i = lane; i < n; i += 32) atomicAdd(&cnt[bin_of_phase(phase_fixed64(t[o0 + i], f), (unsigned)M)], 1u);
    __syncwarp();
    float s = 0.f;
    for (int m = lane; m < M; m += 32) {
      const unsigned q = cnt[m];
      if (q > 1u) s += (float)q * logf((float)q);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) {
      const float N = (float)n;
      const float H = entropy_from_counts_sum(s, N);
      const double Md = (double)M, Nd = (double)n;
      float z = __int_as_float(0x7fc00000);
      if (n > 0 && M > 1) {
        const double E = log(Md) - (Md - 1.0) / (2.0 * Nd) - (Md - 1.0) * (Md + 1.0) / (12.0 * Nd * Nd);
        const double V = (Md - 1.0) / (2.0 * Nd * Nd) + (Md * Md - 1.0) / (6.0 * Nd * Nd * Nd);
        z = (float)(((double)H - E) / sqrt(V));
      }
      H_out[e] = H;
      z_out[e] = z;
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_entropy_dense(const double* t, int64_t n, const double* freqs, int64_t nfreq, int M, float* H_out,
                                 cudaStream_t st) {
  if (nfreq <= 0) return cudaSuccess;
  const size_t smem = (size_t)kEntChunk * 8 + (size_t)M * kEntThreads * 4;
  cudaError_t e = cudaFuncSetAttribute(entropy_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (nfreq + kEntThreads - 1) / kEntThreads;
  entropy_dense_kernel<<<(unsigned)blocks, kEntThreads, smem, st>>>(t, n, freqs, nfreq, M, H_out);
  return cudaGetLastError();
}

cudaError_t launch_entropy_peaks(const int64_t* offsets, int64_t ncurves, const double* t, const double* freqs,
                                 int64_t nfreq, int M, int k, const int32_t* topk_idx, float* H_out, float* z_out,
                                 cudaStream_t st) {
  const int64_t total = ncurves * k;
  if (total <= 0) return cudaSuccess;
  const size_t smem = (size_t)kPeakWarps * M * 4;
  cudaError_t e = cudaFuncSetAttribute(entropy_peaks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t blocks = (total + kPeakWarps - 1) / kPeakWarps;
  blocks = blocks > 65535 ? 65535 : blocks;
  entropy_peaks_kernel<<<(unsigned)blocks, kPeakWarps * 32, smem, st>>>(
      offsets, ncurves, t, freqs, nfreq, M, k, topk_idx, H_out, z_out);
  return cudaGetLastError();
}

}  // namespace fpw
