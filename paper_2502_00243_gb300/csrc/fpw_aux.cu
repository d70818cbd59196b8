// Auxiliary FPW kernels:
//   prep         w_i = 1/sigma_i^2 and a_i = x_i w_i per observation (Eq. 1's
//                weights, computed once per call), input validation
//   merge        per-curve top-k peaks from the per-item candidates (Section 3.5)
//   plain        the binary64 reference form: fl(t f) per evaluation, binary64
//                bins (Appendix A.1) and sums (Eq. 1), one curve per launch
//   dense_topk   top-k peaks of one dense periodogram (for the plain form)
#include <math.h>

#include "fpw_internal.cuh"

namespace fpw {
namespace {

__device__ __forceinline__ int64_t curve_of(const int64_t* offsets, int64_t ncurves, int64_t i) {
  // largest c with offsets[c] <= i (binary search; only used on the error path)
  int64_t lo = 0, hi = ncurves - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__global__ void prep_kernel(const PrepArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.nobs; i += stride) {
    const double s = a.sigma[i], x = a.x[i], t = a.t[i];
    const bool ok = isfinite(s) && isfinite(x) && isfinite(t) && s > 0.0;
    const double w = ok ? 1.0 / (s * s) : 0.0;
    const double xa = ok ? x * w : 0.0;
    if (a.aw == nullptr) {
    } else if (a.accum == FPW_ACCUM_FP64) {
      reinterpret_cast<double2*>(a.aw)[i] = make_double2(xa, w);
    } else if (a.accum == FPW_ACCUM_FP32_COMP) {
      // hi + lo FP32 pairs: the compensated sums add the low parts too
      const float ah = (float)xa, wh = (float)w;
      reinterpret_cast<float4*>(a.aw)[i] = make_float4(ah, wh, (float)(xa - (double)ah), (float)(w - (double)wh));
    } else {
      reinterpret_cast<float2*>(a.aw)[i] = make_float2((float)xa, (float)w);
    }
    if (!ok) {
      const int64_t c = a.offsets ? curve_of(a.offsets, a.ncurves, i) : 0;
      a.curve_bad[c] = 1;
      atomicOr(a.status, kStatusData);
    }
  }
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.nfreq; q += stride)
    if (!isfinite(a.freqs[q])) atomicOr(a.status, kStatusGrid);
}

__device__ __forceinline__ void warp_best(double& bs, int& bi, int& bp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double os = __shfl_xor_sync(0xffffffffu, bs, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    const int op = __shfl_xor_sync(0xffffffffu, bp, o);
    if (op >= 0 && (bp < 0 || ranks_before(os, oi, bs, bi))) {
      bs = os;
      bi = oi;
      bp = op;
    }
  }
}

// One warp per curve: the k best of its candidate rows. A candidate ranks after
// the previously selected one iff it is strictly worse in the (S desc, idx asc)
// order, so no marking is needed.
__global__ void merge_kernel(const MergeArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const bool grid_bad = (*a.status & kStatusGrid) != 0u;
  const int64_t stride = a.out_stride > 0 ? a.out_stride : a.k;
  for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < a.ncurves; c += warps) {
    int32_t* oi = a.topk_idx + c * stride;
    float* os = a.topk_S + c * stride;
    int32_t* oo = a.topk_off ? a.topk_off + c * stride : nullptr;
    if (grid_bad || a.curve_bad[c]) {
      for (int q = lane; q < a.k; q += 32) {
        oi[q] = -1;
        os[q] = __int_as_float(0x7fc00000);
        if (oo) oo[q] = -1;
      }
      continue;
    }
    const int64_t e0 = (int64_t)a.cand_base[c] * a.k, e1 = (int64_t)a.cand_base[c + 1] * a.k;
    double ps = INFINITY;
    int pi = -1;
    for (int q = 0; q < a.k; ++q) {
      double bs = -INFINITY;
      int bi = -1, bp = -1;
      for (int64_t e = e0 + lane; e < e1; e += 32) {
        const int i = a.cand_idx[e];
        if (i < 0) continue;
        const double s = a.cand_S[e];
        const bool after_prev = (q == 0) || ranks_before(ps, pi, s, i);
        if (after_prev && (bp < 0 || ranks_before(s, i, bs, bi))) {
          bs = s;
          bi = i;
          bp = 1;
        }
      }
      warp_best(bs, bi, bp);
      if (lane == 0) {
        if (oo) {
          oi[q] = (bp >= 0) ? (bi >> 6) : -1;
          oo[q] = (bp >= 0) ? (bi & 63) : -1;
        } else {
          oi[q] = (bp >= 0) ? bi : -1;
        }
        os[q] = (bp >= 0) ? (float)bs : __int_as_float(0x7fc00000);
      }
      if (bp < 0) {
        for (int r = q + 1 + lane; r < a.k; r += 32) {
          oi[r] = -1;
          os[r] = __int_as_float(0x7fc00000);
          if (oo) oo[r] = -1;
        }
        break;
      }
      ps = bs;
      pi = bi;
    }
  }
}

// The same selection with one block per curve, for curves with many candidate
// rows (one long curve split into thousands of work items): each round every
// thread scans a slice of the rows and the block reduces the per-warp bests,
// instead of one warp scanning every row k times.
constexpr int kMergeBlock = 256;

__global__ void __launch_bounds__(kMergeBlock) merge_block_kernel(const MergeArgs a) {
  __shared__ double ws[kMergeBlock / 32];
  __shared__ int wi[kMergeBlock / 32];
  __shared__ int wp[kMergeBlock / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool grid_bad = (*a.status & kStatusGrid) != 0u;
  const int64_t stride = a.out_stride > 0 ? a.out_stride : a.k;
  for (int64_t c = blockIdx.x; c < a.ncurves; c += gridDim.x) {
    int32_t* oi = a.topk_idx + c * stride;
    float* os = a.topk_S + c * stride;
    int32_t* oo = a.topk_off ? a.topk_off + c * stride : nullptr;
    if (grid_bad || a.curve_bad[c]) {
      for (int q = tid; q < a.k; q += kMergeBlock) {
        oi[q] = -1;
        os[q] = __int_as_float(0x7fc00000);
        if (oo) oo[q] = -1;
      }
      continue;
    }
    const int64_t e0 = (int64_t)a.cand_base[c] * a.k, e1 = (int64_t)a.cand_base[c + 1] * a.k;
    double ps = INFINITY;
    int pi = -1;
    for (int q = 0; q < a.k; ++q) {
      double bs = -INFINITY;
      int bi = -1, bp = -1;
      for (int64_t e = e0 + tid; e < e1; e += kMergeBlock) {
        const int i = a.cand_idx[e];
        if (i < 0) continue;
        const double s = a.cand_S[e];
        const bool after_prev = (q == 0) || ranks_before(ps, pi, s, i);
        if (after_prev && (bp < 0 || ranks_before(s, i, bs, bi))) {
          bs = s;
          bi = i;
          bp = 1;
        }
      }
      warp_best(bs, bi, bp);
      if (lane == 0) {
        ws[warp] = bs;
        wi[warp] = bi;
        wp[warp] = bp;
      }
      __syncthreads();
      if (warp == 0) {
        bs = lane < kMergeBlock / 32 ? ws[lane] : -INFINITY;
        bi = lane < kMergeBlock / 32 ? wi[lane] : -1;
        bp = lane < kMergeBlock / 32 ? wp[lane] : -1;
        warp_best(bs, bi, bp);
        if (lane == 0) {
          if (oo) {
            oi[q] = (bp >= 0) ? (bi >> 6) : -1;
            oo[q] = (bp >= 0) ? (bi & 63) : -1;
          } else {
            oi[q] = (bp >= 0) ? bi : -1;
          }
          os[q] = (bp >= 0) ? (float)bs : __int_as_float(0x7fc00000);
          ws[0] = bs;
          wi[0] = bi;
          wp[0] = bp;
        }
      }
      __syncthreads();
      ps = ws[0];
      pi = wi[0];
      const bool none = wp[0] < 0;
      __syncthreads();
      if (none) {
        for (int r = q + 1 + tid; r < a.k; r += kMergeBlock) {
          oi[r] = -1;
          os[r] = __int_as_float(0x7fc00000);
          if (oo) oo[r] = -1;
        }
        break;
      }
    }
  }
}

// Plain binary64 form. One thread per trial frequency; observations staged in
// shared memory in chunks; per-thread bins [m][thread] as {A, B} binary64.
// DUMP: also writes the bin of every (observation, frequency) in the window.
constexpr int kPlainThreads = 128;
constexpr int kPlainChunk = 256;

template <bool DUMP>
__global__ void __launch_bounds__(kPlainThreads) plain_kernel(const PlainArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* st = reinterpret_cast<double*>(smem);
  double* sa = st + kPlainChunk;
  double* sw = sa + kPlainChunk;
  double2* bins = reinterpret_cast<double2*>(sw + kPlainChunk);
  const int tid = threadIdx.x;
  const int64_t k = (int64_t)blockIdx.x * kPlainThreads + tid;
  const double f = a.freqs[k < a.nfreq ? k : a.nfreq - 1];
  const int M = a.M;
  for (int m = 0; m < M; ++m) bins[m * kPlainThreads + tid] = make_double2(0.0, 0.0);
  bool bad = false;
  for (int64_t o = 0; o < a.n; o += kPlainChunk) {
    const int cnt = (int)((a.n - o) < kPlainChunk ? (a.n - o) : kPlainChunk);
    __syncthreads();
    for (int i = tid; i < cnt; i += kPlainThreads) {
      const double s = a.sigma[o + i], x = a.x[o + i], t = a.t[o + i];
      if (!(isfinite(s) && isfinite(x) && isfinite(t) && s > 0.0)) bad = true;
      const double w = 1.0 / (s * s);
      st[i] = t;
      sa[i] = x * w;
      sw[i] = w;
    }
    __syncthreads();
    for (int i = 0; i < cnt; ++i) {
      const double p = __dmul_rn(st[i], f);
      const double ph = __dsub_rn(p, floor(p));
      int m = (int)floor(__dmul_rn((double)M, ph));
      m = m > M - 1 ? M - 1 : (m < 0 ? 0 : m);
      if (DUMP && k < a.nfreq && k >= a.bins_k0 && k < a.bins_k1)
        a.bins_out[(k - a.bins_k0) * a.bins_nobs + a.bins_base + o + i] = m;
      double2* b = &bins[m * kPlainThreads + tid];
      double2 v = *b;
      v.x = __dadd_rn(v.x, sa[i]);
      v.y = __dadd_rn(v.y, sw[i]);
      *b = v;
    }
  }
  bad = __syncthreads_or(bad);
  if (bad && tid == 0) atomicOr(a.status, kStatusData);
  if (k < a.nfreq) {
    double S = 0.0;
    for (int m = 0; m < M; ++m) {
      const double2 v = bins[m * kPlainThreads + tid];
      const double den = __dadd_rn(v.y, a.inv_alpha2);
      if (den > 0.0) S = __dadd_rn(S, __ddiv_rn(__dmul_rn(v.x, v.x), den));
    }
    a.S_out[k] = bad ? __longlong_as_double(0x7ff8000000000000ll) : S;
  }
}

// Top-k peaks of one dense periodogram, one block: k rounds of a block-wide
// arg-max restricted to entries ranked strictly after the previous pick.
constexpr int kTopkThreads = 1024;

__global__ void __launch_bounds__(kTopkThreads) dense_topk_kernel(const DenseTopkArgs a) {
  __shared__ double ws[32];
  __shared__ int wi[32];
  __shared__ int wp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t F = a.nfreq;
  const bool bad = F > 0 && isnan(a.S[0]);  // the plain kernel writes NaN for invalid curves
  double ps = INFINITY;
  int pi = -1;
  for (int q = 0; q < a.k; ++q) {
    double bs = -INFINITY;
    int bi = -1, bp = -1;
    if (!bad) {
      for (int64_t e = tid; e < F; e += kTopkThreads) {
        const double s = a.S[e];
        bool peak = true;
        if (!a.peak_raw) {
          const double l = (e > 0) ? a.S[e - 1] : -INFINITY;
          const double r = (e + 1 < F) ? a.S[e + 1] : -INFINITY;
          peak = s > l && s >= r;
        }
        if (!peak) continue;
        const bool after_prev = (q == 0) || ranks_before(ps, pi, s, (int)e);
        if (after_prev && (bp < 0 || ranks_before(s, (int)e, bs, bi))) {
          bs = s;
          bi = (int)e;
          bp = 1;
        }
      }
    }
    warp_best(bs, bi, bp);
    if (lane == 0) {
      ws[warp] = bs;
      wi[warp] = bi;
      wp[warp] = bp;
    }
    __syncthreads();
    if (warp == 0) {
      bs = ws[lane];
      bi = wi[lane];
      bp = wp[lane];
      warp_best(bs, bi, bp);
      if (lane == 0) {
        a.topk_idx[q] = (bp >= 0) ? bi : -1;
        a.topk_S[q] = (bp >= 0) ? (float)bs : __int_as_float(0x7fc00000);
        wi[0] = bi;
        wp[0] = bp;
        ws[0] = bs;
      }
    }
    __syncthreads();
    ps = ws[0];
    pi = wi[0];
    if (wp[0] < 0) {
      for (int r = q + 1 + tid; r < a.k; r += kTopkThreads) {
        a.topk_idx[r] = -1;
        a.topk_S[r] = __int_as_float(0x7fc00000);
      }
      break;
    }
    __syncthreads();
  }
}

__global__ void latch_kernel(unsigned* words) { words[2] |= words[1]; }

__global__ void fill_topk_kernel(int32_t* idx, float* S, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    idx[i] = -1;
    S[i] = __int_as_float(0x7fc00000);
  }
}

}  // namespace

cudaError_t launch_latch(unsigned* words, cudaStream_t st) {
  latch_kernel<<<1, 1, 0, st>>>(words);
  return cudaGetLastError();
}

cudaError_t launch_fill_topk(int32_t* idx, float* S, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  blocks = blocks > 4096 ? 4096 : blocks;
  fill_topk_kernel<<<(unsigned)blocks, 256, 0, st>>>(idx, S, n);
  return cudaGetLastError();
}

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t st) {
  const int64_t work = a.nobs > a.nfreq ? a.nobs : a.nfreq;
  int blocks = (int)((work + 255) / 256);
  blocks = blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks);
  prep_kernel<<<blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_merge(const MergeArgs& a, cudaStream_t st) {
  if (a.ncurves <= 0 || a.k <= 0) return cudaSuccess;
  if ((int64_t)a.max_rows * a.k > 512) {  // long curves: a block per curve
    const int64_t blocks = a.ncurves < 65535 ? a.ncurves : 65535;
    merge_block_kernel<<<(unsigned)blocks, kMergeBlock, 0, st>>>(a);
    return cudaGetLastError();
  }
  int blocks = (int)((a.ncurves + 7) / 8);
  blocks = blocks > 65535 ? 65535 : blocks;
  merge_kernel<<<blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

size_t plain_smem_bytes(int M) { return (size_t)3 * kPlainChunk * 8 + (size_t)M * kPlainThreads * 16; }

cudaError_t plain_init_attributes(int max_smem) {
  cudaError_t e = cudaFuncSetAttribute(plain_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(plain_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

cudaError_t launch_plain(const PlainArgs& a, cudaStream_t st) {
  if (a.nfreq <= 0) return cudaSuccess;
  const size_t smem = plain_smem_bytes(a.M);
  const int64_t blocks = (a.nfreq + kPlainThreads - 1) / kPlainThreads;
  if (a.bins_out)
    plain_kernel<true><<<(unsigned)blocks, kPlainThreads, smem, st>>>(a);
  else
    plain_kernel<false><<<(unsigned)blocks, kPlainThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dense_topk(const DenseTopkArgs& a, cudaStream_t st) {
  if (a.k <= 0) return cudaSuccess;
  dense_topk_kernel<<<1, kTopkThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace fpw
