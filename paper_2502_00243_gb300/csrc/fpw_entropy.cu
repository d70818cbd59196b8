// Phase entropy of the observation times (Appendix C):
//   H(f) = -sum_m (N_m / N) log(N_m / N),  N_m observations in phase bin m,
// with Hutcheson's expectation and variance for equally likely bins,
//   E(H)   = log M - (M - 1) / (2 N) - (M - 1)(M + 1) / (12 N^2),
//   Var(H) = (M - 1) / (2 N^2) + (M^2 - 1) / (6 N^3),
// used to flag periodogram peaks whose phase coverage is anomalously uneven
// (z = (H - E) / sqrt(Var) strongly negative).
//
// Bins use the exact anchors and 64-bit stepping of the periodogram kernels,
// so they equal floor(M frac(t f)) except within 2e-10 cycles of an edge.
#include <math.h>

#include "fpw_internal.cuh"

namespace fpw {
namespace {

constexpr int kEntThreads = 128;
constexpr int kEntChunk = 256;

// H from bin counts: log N - (1/N) sum_m N_m log N_m, in FP32 (the count
// terms are exact integers; the logarithms carry the rounding).
__device__ __forceinline__ float entropy_from_counts_sum(float sum_clogc, float N) {
  return N > 0.f ? logf(N) - sum_clogc / N : 0.f;
}

// R consecutive frequencies per thread, blocks of kEntThreads R frequencies;
// counts per (frequency slot, bin, thread) as 32-bit integers, [r][m][thread]
// (conflict-free). Per staged observation the block holds the exact anchor
// phase at its first frequency, P_i = frac(t_i f_0), and the step D_i =
// frac(t_i df) as 64-bit fixed point; where the block's frequencies lie on the
// linear grid (the tile kernels' bound on the phase error) frequency j of the
// block has phase P_i + j D_i (mod 2^64), as in the periodogram kernels, else
// the exact anchor at its own frequency. One observation per iteration: its R
// counts (in disjoint slots) are all loaded before any store, and the next
// observation's staged data is loaded before them.
template <int R>
__global__ void __launch_bounds__(kEntThreads) entropy_dense_kernel(const double* t, int64_t n, const double* freqs,
                                                                    int64_t nfreq, int M, float* H_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  ulonglong2* const sPD = reinterpret_cast<ulonglong2*>(smem);
  unsigned* const cnt = reinterpret_cast<unsigned*>(sPD + kEntChunk + 1);  // one record of padding after the chunk
  __shared__ double s_tm[kEntThreads / 32];
  const int tid = threadIdx.x;
  const int64_t f0 = (int64_t)blockIdx.x * (kEntThreads * R);
  const int j0 = tid * R;  // the thread's first frequency within the block
  const double fa = freqs[f0];
  const double df = (nfreq > 1) ? (freqs[nfreq - 1] - freqs[0]) / (double)(nfreq - 1) : 0.0;
  double fk[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t k = f0 + j0 + r;
    fk[r] = freqs[k < nfreq ? k : nfreq - 1];
  }
  double tm = 0.0;
  for (int64_t i = tid; i < n; i += kEntThreads) tm = fmax(tm, fabs(t[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tm = fmax(tm, __shfl_xor_sync(0xffffffffu, tm, o));
  if ((tid & 31) == 0) s_tm[tid >> 5] = tm;
  __syncthreads();
  tm = 0.0;
#pragma unroll
  for (int q = 0; q < kEntThreads / 32; ++q) tm = fmax(tm, s_tm[q]);
  bool nonlin = false;
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (f0 + j0 + r < nfreq && fabs(fk[r] - fma((double)(j0 + r), df, fa)) * tm > kGridTolCycles) nonlin = true;
  const bool lin = !__syncthreads_or(nonlin);
  const int MT = M * kEntThreads;
  for (int q = 0; q < R * M; ++q) cnt[q * kEntThreads + tid] = 0u;
  for (int64_t o = 0; o < n; o += kEntChunk) {
    const int c = (int)((n - o) < kEntChunk ? (n - o) : kEntChunk);
    __syncthreads();
    for (int i = tid; i < c; i += kEntThreads) {
      const double ti = t[o + i];
      sPD[i] = lin ? make_ulonglong2(phase_fixed64(ti, fa), phase_fixed64(ti, df))
                   : make_ulonglong2((unsigned long long)__double_as_longlong(ti), 0ull);
    }
    if (tid == 0) sPD[c] = make_ulonglong2(0ull, 0ull);  // read by the last iteration's prefetch, never used
    __syncthreads();
    unsigned* const mine = cnt + tid;  // this thread's column of the [r][m][thread] counts
    if (lin) {
      ulonglong2 pd = sPD[0];
#pragma unroll 2
      for (int i = 0; i < c; ++i) {
        const ulonglong2 pdn = sPD[i + 1];  // i + 1 <= c <= kEntChunk: staged or the zeroed record
        // the R phases are independent multiply-adds (no serial chain of 64-bit adds)
        const unsigned long long phi0 = pd.x + (unsigned long long)j0 * pd.y;
        unsigned* sl[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
          sl[r] = mine + r * MT + bin_of_phase(phi0 + (unsigned long long)r * pd.y, (unsigned)M) * kEntThreads;
        unsigned v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = *sl[r];
#pragma unroll
        for (int r = 0; r < R; ++r) *sl[r] = v[r] + 1u;
        pd = pdn;
      }
    } else {
      for (int i = 0; i < c; ++i) {
        const double ti = __longlong_as_double((long long)sPD[i].x);
        unsigned* sl[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
          sl[r] = mine + r * MT + bin_of_phase(phase_fixed64(ti, fk[r]), (unsigned)M) * kEntThreads;
        unsigned v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = *sl[r];
#pragma unroll
        for (int r = 0; r < R; ++r) *sl[r] = v[r] + 1u;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t k = f0 + j0 + r;
    if (k < nfreq) {
      float s = 0.f;
      for (int m = 0; m < M; ++m) {
        const unsigned q = cnt[r * MT + m * kEntThreads + tid];
        if (q > 1u) s += (float)q * logf((float)q);
      }
      H_out[k] = entropy_from_counts_sum(s, (float)n);
    }
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
  // frequencies per thread: as many as keep the counts of a block within
  // 48 KB (four blocks per SM), one beyond M = 96. Measured on the N = 1000
  // ZTF-cadence times over 1e6 frequencies: M = 10 2.75e12 evaluations/s at
  // R = 8 against 2.62e12 at R = 4; M = 20 2.54e12 at R = 4 against 2.08e12 at
  // R = 8 (two blocks per SM). 16-bit counts (twice the blocks per SM) ran
  // slower at every M (M = 20, R = 4: 2.07e12).
  const int R = M <= 12 ? 8 : (M <= 24 ? 4 : (M <= 96 ? 2 : 1));
  const void* fn = R == 8   ? reinterpret_cast<const void*>(&entropy_dense_kernel<8>)
                   : R == 4 ? reinterpret_cast<const void*>(&entropy_dense_kernel<4>)
                   : R == 2 ? reinterpret_cast<const void*>(&entropy_dense_kernel<2>)
                            : reinterpret_cast<const void*>(&entropy_dense_kernel<1>);
  const size_t smem = (size_t)(kEntChunk + 1) * 16 + (size_t)R * M * kEntThreads * 4;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t per_block = (int64_t)kEntThreads * R;
  const int64_t blocks = (nfreq + per_block - 1) / per_block;
  void* args[] = {const_cast<double**>(&t), &n, const_cast<double**>(&freqs), &nfreq, &M, &H_out};
  return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(kEntThreads), args, smem, st);
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
