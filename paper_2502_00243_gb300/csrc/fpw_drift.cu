// FPW with the baseline drift marginalised (Appendix A.1-A.2) for a ragged
// batch: the covariance of the data is C_B + C_sigma, C_B = B B^T with a
// Chebyshev basis B[i, k] = beta T_k(tau_i), k < K (tau: the curve's times
// mapped to [-1, 1]), and the statistic is
//
//   S = u^T (I / alpha^2 + E^T W E)^-1 u,   u = E^T W x,   W = (C_B + C_sigma)^-1.
//
// With D = diag(w), H0 = I + B^T D B and g = H0^-1 B^T D x (per curve, once),
// Woodbury twice reduces it to per-bin sums over the observations in bin m,
//
//   Y_m = sum w x,   Bw_m = sum w,   Q_mk = sum w B_ik,
//
// and a K x K system per frequency:
//
//   z_m = Y_m - Q_m . g,  L_m = Bw_m + 1/alpha^2,
//   S = sum_m z_m^2 / L_m + v^T H^-1 v,  v = sum_m Q_m z_m / L_m,
//   H = H0 - sum_m Q_m Q_m^T / L_m   (symmetric positive definite, >= I).
//
// Bins with no observation and 1/alpha^2 = 0 are dropped (their rows vanish).
// The sums accumulate in FP32 in thread-private shared-memory bins (one thread
// per frequency, (2 + K) floats per bin, packed), phases are the exact 64-bit anchors
// of the tile kernels stepped across a tile of frequencies; the per-frequency
// reduction and the K x K Cholesky solve run in binary64.
#include <math.h>

#include "fpw_shared.cuh"

namespace fpw {
namespace {

constexpr int kDrMaxK = 4;
constexpr int kDrPay = 2 + kDrMaxK;  // payload floats per observation: w x, w, w B_0..B_{K-1}
constexpr int kDrChunk = 256;        // observations staged at a time

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per curve (one block of 256 threads): validation, the time span, the payload
// of every observation, H0 = I + B^T D B and g = H0^-1 B^T D x.
__global__ void __launch_bounds__(256) drift_prep_kernel(const DriftArgs a) {
  __shared__ double red[8][kDrMaxK * kDrMaxK + kDrMaxK + 3];
  __shared__ double tl[2];
  const int64_t c = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = a.K;
  const int64_t o0 = a.offsets[c], n = a.offsets[c + 1] - o0;
  // validation and the time span
  double tmin = INFINITY, tmax = -INFINITY;
  int bad = 0;
  for (int64_t i = tid; i < n; i += blockDim.x) {
    const double s = a.sigma[o0 + i], x = a.x[o0 + i], t = a.t[o0 + i];
    if (!(isfinite(s) && isfinite(x) && isfinite(t) && s > 0.0)) bad = 1;
    if (isfinite(t)) {
      tmin = fmin(tmin, t);
      tmax = fmax(tmax, t);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
    tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (lane == 0) {
    red[warp][0] = tmin;
    red[warp][1] = tmax;
    red[warp][2] = (double)bad;
  }
  __syncthreads();
  if (tid == 0) {
    double a0 = INFINITY, a1 = -INFINITY, b = 0.0;
    for (int q = 0; q < 8; ++q) {
      a0 = fmin(a0, red[q][0]);
      a1 = fmax(a1, red[q][1]);
      b = fmax(b, red[q][2]);
    }
    tl[0] = a0;
    tl[1] = a1;
    a.curve_bad[c] = b > 0.0 ? 1 : 0;
    if (b > 0.0) atomicOr(a.status, kStatusData);
  }
  __syncthreads();
  const bool cbad = a.curve_bad[c] != 0;
  const double lo = tl[0], span = tl[1] - tl[0];
  // payload and the curve sums B^T D B (K x K) and B^T D x (K)
  double acc[kDrMaxK * kDrMaxK + kDrMaxK];
#pragma unroll
  for (int q = 0; q < kDrMaxK * kDrMaxK + kDrMaxK; ++q) acc[q] = 0.0;
  for (int64_t i = tid; i < n; i += blockDim.x) {
    float* pay = a.payload + (size_t)(o0 + i) * kDrPay;
    double w = 0.0, x = 0.0;
    if (!cbad) {
      const double s = a.sigma[o0 + i];
      w = 1.0 / (s * s);
      x = a.x[o0 + i];
    }
    const double tau = (span > 0.0) ? 2.0 * (a.t[o0 + i] - lo) / span - 1.0 : 0.0;
    double Bk[kDrMaxK];
    double tkm1 = 1.0, tk = tau;
#pragma unroll
    for (int k = 0; k < kDrMaxK; ++k) {
      double T;
      if (k == 0) {
        T = 1.0;
      } else if (k == 1) {
        T = tau;
      } else {
        const double tn = 2.0 * tau * tk - tkm1;
        tkm1 = tk;
        tk = tn;
        T = tn;
      }
      Bk[k] = a.beta * T;
    }
    pay[0] = (float)(w * x);
    pay[1] = (float)w;
#pragma unroll
    for (int k = 0; k < kDrMaxK; ++k) {
      pay[2 + k] = k < K ? (float)(w * Bk[k]) : 0.f;
      if (k < K) {
#pragma unroll
        for (int l = 0; l < kDrMaxK; ++l)
          if (l < K) acc[k * kDrMaxK + l] += w * Bk[k] * Bk[l];
        acc[kDrMaxK * kDrMaxK + k] += w * Bk[k] * x;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kDrMaxK * kDrMaxK + kDrMaxK; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double H[kDrMaxK][kDrMaxK], r[kDrMaxK];
    for (int k = 0; k < K; ++k) {
      r[k] = 0.0;
      for (int l = 0; l < K; ++l) {
        double s = 0.0;
        for (int q = 0; q < 8; ++q) s += red[q][k * kDrMaxK + l];
        H[k][l] = s + (k == l ? 1.0 : 0.0);
      }
      for (int q = 0; q < 8; ++q) r[k] += red[q][kDrMaxK * kDrMaxK + k];
    }
    double* h0 = a.H0 + c * kDrMaxK * kDrMaxK;
    for (int k = 0; k < kDrMaxK * kDrMaxK; ++k) h0[k] = (k / kDrMaxK < K && k % kDrMaxK < K) ? H[k / kDrMaxK][k % kDrMaxK] : 0.0;
    // g = H0^-1 B^T D x by Cholesky (H0 >= I is positive definite)
    double Lc[kDrMaxK][kDrMaxK];
    for (int k = 0; k < K; ++k)
      for (int l = 0; l <= k; ++l) {
        double s = H[k][l];
        for (int q = 0; q < l; ++q) s -= Lc[k][q] * Lc[l][q];
        Lc[k][l] = (k == l) ? sqrt(s) : s / Lc[l][l];
      }
    double y[kDrMaxK];
    for (int k = 0; k < K; ++k) {
      double s = r[k];
      for (int q = 0; q < k; ++q) s -= Lc[k][q] * y[q];
      y[k] = s / Lc[k][k];
    }
    double* g = a.g + c * kDrMaxK;
    for (int k = K - 1; k >= 0; --k) {
      double s = y[k];
      for (int q = k + 1; q < K; ++q) s -= Lc[q][k] * g[q];
      g[k] = s / Lc[k][k];
    }
    for (int k = K; k < kDrMaxK; ++k) g[k] = 0.0;
  }
  if (blockIdx.x == 0)
    for (int64_t q = tid; q < a.nfreq; q += blockDim.x)
      if (!isfinite(a.freqs[q])) atomicOr(a.status, kStatusGrid);
}

// One block per (tile of T frequencies, curve); thread = frequency. Bins
// thread-private (bank = lane): (Y, Bw) as float2 [M][T] and, for K > 0, the
// K sums w B_k as float4 [M][T]: two packed read-modify-writes per evaluation,
// loads issued before stores.
template <int K>
__global__ void __launch_bounds__(128) drift_kernel(const DriftArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, tid = threadIdx.x;
  const int M = a.M;
  const int64_t c = blockIdx.y, F = a.nfreq;
  const int64_t f0 = (int64_t)blockIdx.x * T, k = f0 + tid;
  float2* bYB = reinterpret_cast<float2*>(smem);                               // [M][T]
  float4* bQ = reinterpret_cast<float4*>(bYB + (size_t)M * T);                  // [M][T] (K > 0)
  ulonglong2* sPD = reinterpret_cast<ulonglong2*>(bQ + (K > 0 ? (size_t)M * T : 0));  // [chunk]
  float2* sYB = reinterpret_cast<float2*>(sPD + kDrChunk);                      // [chunk]
  float4* sQ = reinterpret_cast<float4*>(sYB + kDrChunk);                       // [chunk]
  const bool grid_bad = (*(volatile unsigned*)a.status & kStatusGrid) != 0u;
  if (grid_bad) return;
  const bool cbad = a.curve_bad[c] != 0;
  const int64_t o0 = a.offsets[c], n = a.offsets[c + 1] - o0;
  const double df = (F > 1) ? (a.freqs[F - 1] - a.freqs[0]) / (double)(F - 1) : 0.0;
  const double fa = a.freqs[f0];
  // linear grid over this tile (the tile kernels' bound on the phase error)?
  double tm = 0.0;
  for (int64_t i = tid; i < n; i += T) tm = fmax(tm, fabs(a.t[o0 + i]));
  __shared__ double s_tm[4];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tm = fmax(tm, __shfl_xor_sync(0xffffffffu, tm, o));
  if ((tid & 31) == 0) s_tm[tid >> 5] = tm;
  __syncthreads();
  tm = 0.0;
  for (int q = 0; q < (T >> 5); ++q) tm = fmax(tm, s_tm[q]);
  const double fk = k < F ? a.freqs[k] : fa;
  const bool nonlin = k < F && fabs(fk - fma((double)tid, df, fa)) * tm > kGridTolCycles;
  const bool lin = !__syncthreads_or(nonlin);
  for (int m = 0; m < M; ++m) {
    bYB[m * T + tid] = make_float2(0.f, 0.f);
    if (K > 0) bQ[m * T + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int64_t oc = 0; oc < n; oc += kDrChunk) {
    const int cnt = (int)((n - oc) < kDrChunk ? (n - oc) : kDrChunk);
    __syncthreads();
    for (int i = tid; i < cnt; i += T) {
      const double ti = a.t[o0 + oc + i];
      sPD[i] = lin ? make_ulonglong2(phase_fixed64(ti, fa), phase_fixed64(ti, df))
                   : make_ulonglong2((unsigned long long)__double_as_longlong(ti), 0ull);
      const float* pay = a.payload + (size_t)(o0 + oc + i) * kDrPay;
      sYB[i] = make_float2(pay[0], pay[1]);
      if (K > 0) sQ[i] = make_float4(pay[2], pay[3], pay[4], pay[5]);
    }
    __syncthreads();
    if (!cbad) {
      float2* const yb = bYB + tid;
      float4* const qb = bQ + tid;
      auto bin_T = [&](const ulonglong2 pd) {
        const unsigned long long phi =
            lin ? pd.x + (unsigned long long)tid * pd.y : phase_fixed64(__longlong_as_double((long long)pd.x), fk);
        return (int)bin_of_phase(phi, (unsigned)M) * T;
      };
      // two observations per iteration: both read-modify-write chains are in
      // flight at once; where both fall in one bin the second update starts
      // from the first one's sum (same additions in the same order)
      int i = 0;
      for (; i + 1 < cnt; i += 2) {
        const int ma = bin_T(sPD[i]), mb = bin_T(sPD[i + 1]);
        const float2 pa = sYB[i], pb = sYB[i + 1];
        float2 va = yb[ma], vb = yb[mb];
        float4 qa, qbv;
        if (K > 0) {
          qa = qb[ma];
          qbv = qb[mb];
        }
        const float2 ua = make_float2(va.x + pa.x, va.y + pa.y);
        if (ma == mb) vb = ua;
        yb[ma] = ua;
        yb[mb] = make_float2(vb.x + pb.x, vb.y + pb.y);
        if (K > 0) {
          const float4 ra = sQ[i], rb = sQ[i + 1];
          const float4 wa = make_float4(qa.x + ra.x, qa.y + ra.y, qa.z + ra.z, qa.w + ra.w);
          if (ma == mb) qbv = wa;
          qb[ma] = wa;
          qb[mb] = make_float4(qbv.x + rb.x, qbv.y + rb.y, qbv.z + rb.z, qbv.w + rb.w);
        }
      }
      if (i < cnt) {
        const int mT = bin_T(sPD[i]);
        const float2 p2 = sYB[i];
        const float2 v2 = yb[mT];
        yb[mT] = make_float2(v2.x + p2.x, v2.y + p2.y);
        if (K > 0) {
          const float4 v4 = qb[mT], p4 = sQ[i];
          qb[mT] = make_float4(v4.x + p4.x, v4.y + p4.y, v4.z + p4.z, v4.w + p4.w);
        }
      }
    }
  }
  if (k >= F) return;
  // binary64 reduction: S = sum z^2 / L + v^T H^-1 v
  double H[kDrMaxK][kDrMaxK], v[kDrMaxK], g[kDrMaxK];
  const double* h0 = a.H0 + c * kDrMaxK * kDrMaxK;
#pragma unroll
  for (int p = 0; p < K; ++p) {
    g[p] = a.g[c * kDrMaxK + p];
    v[p] = 0.0;
#pragma unroll
    for (int q = 0; q < K; ++q) H[p][q] = h0[p * kDrMaxK + q];
  }
  const double cal = a.inv_alpha2;
  double S = 0.0;
  for (int m = 0; m < M; ++m) {
    const float2 yb = bYB[m * T + tid];
    const double L = (double)yb.y + cal;
    if (!(L > 0.0)) continue;  // empty bin with 1/alpha^2 = 0: dropped
    double Q[kDrMaxK];
    double z = yb.x;
    if (K > 0) {
      const float4 q4 = bQ[m * T + tid];
      const float qq[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
      for (int p = 0; p < K; ++p) {
        Q[p] = qq[p];
        z -= Q[p] * g[p];
      }
    }
    const double zl = z / L;
    S += z * zl;
#pragma unroll
    for (int p = 0; p < K; ++p) {
      v[p] += Q[p] * zl;
#pragma unroll
      for (int q = 0; q < K; ++q) H[p][q] -= Q[p] * Q[q] / L;
    }
  }
  // v^T H^-1 v by Cholesky (H >= I)
  double Lc[kDrMaxK][kDrMaxK], y[kDrMaxK];
#pragma unroll
  for (int p = 0; p < K; ++p)
#pragma unroll
    for (int q = 0; q <= p; ++q) {
      double s = H[p][q];
#pragma unroll
      for (int r = 0; r < q; ++r) s -= Lc[p][r] * Lc[q][r];
      Lc[p][q] = (p == q) ? sqrt(s > 0.0 ? s : 0.0) : s / Lc[q][q];
    }
#pragma unroll
  for (int p = 0; p < K; ++p) {
    double s = v[p];
#pragma unroll
    for (int r = 0; r < p; ++r) s -= Lc[p][r] * y[r];
    y[p] = Lc[p][p] > 0.0 ? s / Lc[p][p] : 0.0;
    S += y[p] * y[p];
  }
  const float Sf = cbad ? __int_as_float(0x7fc00000) : (float)S;
  if (a.S32) a.S32[c * F + k] = Sf;
  if (a.S_out) a.S_out[c * F + k] = cbad ? (double)Sf : S;
}

const void* drift_fn(int K) {
  switch (K) {
    case 0: return reinterpret_cast<const void*>(&drift_kernel<0>);
    case 1: return reinterpret_cast<const void*>(&drift_kernel<1>);
    case 2: return reinterpret_cast<const void*>(&drift_kernel<2>);
    case 3: return reinterpret_cast<const void*>(&drift_kernel<3>);
    default: return reinterpret_cast<const void*>(&drift_kernel<4>);
  }
}

}  // namespace

// Dynamic shared memory the drift kernel may use: the opt-in limit minus its
// static shared memory.
static size_t drift_dynamic_limit(int smem_optin) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, drift_fn(4)) != cudaSuccess) return 0;
  return smem_optin > (int)fa.sharedSizeBytes ? (size_t)(smem_optin - (int)fa.sharedSizeBytes) : 0;
}

int drift_threads(int M, int K, int smem_optin) {
  const size_t lim = drift_dynamic_limit(smem_optin);
  for (int T = 128; T >= 32; T >>= 1)
    if (drift_smem_bytes(M, K, T) <= lim) return T;
  return 0;
}

size_t drift_smem_bytes(int M, int K, int T) {
  return (size_t)M * T * (K > 0 ? 24 : 8) + (size_t)kDrChunk * (16 + 8 + 16);
}

int drift_max_basis() { return kDrMaxK; }

int drift_payload_floats() { return kDrPay; }

cudaError_t drift_init_attributes(int max_smem) {
  const int lim = (int)drift_dynamic_limit(max_smem);
  for (int K = 0; K <= kDrMaxK; ++K) {
    const cudaError_t e = cudaFuncSetAttribute(drift_fn(K), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_drift(const DriftArgs& a, int T, cudaStream_t st) {
  if (a.ncurves <= 0) return cudaSuccess;
  drift_prep_kernel<<<(unsigned)a.ncurves, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.nfreq <= 0) return e;
  const int64_t tiles = (a.nfreq + T - 1) / T;
  if (a.timing_start) cudaEventRecord(a.timing_start, st);
  void* params[] = {const_cast<DriftArgs*>(&a)};
  e = cudaLaunchKernel(drift_fn(a.K), dim3((unsigned)tiles, (unsigned)a.ncurves), dim3(T), params,
                       drift_smem_bytes(a.M, a.K, T), st);
  if (e != cudaSuccess) return e;
  if (a.timing_stop) cudaEventRecord(a.timing_stop, st);
  if (a.k > 0) {
    DenseTopk32Args t{};
    t.S32 = a.S32;
    t.nfreq = a.nfreq;
    t.k = a.k;
    t.peak_raw = a.peak_raw;
    t.curve_bad = a.curve_bad;
    t.status = a.status;
    t.topk_idx = a.topk_idx;
    t.topk_S = a.topk_S;
    e = launch_dense_topk32(t, a.ncurves, st);
  }
  return e;
}

}  // namespace fpw
