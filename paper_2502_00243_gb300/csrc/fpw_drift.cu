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
// Since z_m = sum over bin m of w (x - B g), the bins accumulate the residuals
// of the baseline fit (formed per observation in binary64) and hold z_m
// itself: a drift far above the noise never enters an FP32 sum. B_0 = beta T_0
// = beta is constant, so Q_m0 = beta Bw_m needs no sum of its own: a bin holds
// z, Bw and Q_m1..Q_m(K-1), 1 + max(K, 1) floats; the row of H and the entry of
// v that belong to B_0 take closed forms in the bin sums.
// The sums accumulate in FP32 in thread-private shared-memory bins (one thread
// per frequency, packed as float2 / float4 / float4 + float), phases are the
// exact 64-bit anchors of the tile kernels stepped across a tile of
// frequencies; the per-frequency reduction (one reciprocal per bin, the lower
// triangle of the symmetric H) and the K x K Cholesky solve run in binary64.
#include <math.h>

#include "fpw_shared.cuh"

namespace fpw {
namespace {

constexpr int kDrMaxK = 4;
constexpr int kDrChunk = 128;  // observations staged at a time

// Per observation, written once by the prep kernel.
struct DriftObs {
  float4 q;                // w (x - B g) (w x for K = 0), w, w B_1, w B_2
  unsigned long long D;    // frac(t df) as 64-bit fixed point (linear grids)
  float q3;                // w B_3
  float pad;
};
static_assert(sizeof(DriftObs) == 32, "32-byte records");

// Bytes of the staged copy of one observation: {Phi, D}, q and, for K = 4, q3.
__host__ __device__ constexpr int drift_stage_bytes(int K) { return 16 + 16 + (K > 3 ? 4 : 0); }
// Bytes of one (frequency, bin) slot: (Y, Bw), then Q_1, Q_2 in the same
// float4 for K = 2, 3, and Q_3 in a float of its own for K = 4.
__host__ __device__ constexpr int drift_bin_bytes(int K) { return K <= 1 ? 8 : (K <= 3 ? 16 : 20); }

// float -> double from the IEEE 754 layouts with integer operations (exact for
// normal numbers and zero; subnormal, infinite and NaN inputs take the
// hardware conversion).
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) {
    if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
  }
  const unsigned hi = ((u & 0x80000000u) | ((u & 0x7FFFFFFFu) >> 3)) + (896u << 20);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// 1/L in binary64 from the FP32 reciprocal of Lf (L formed in FP32) and one
// Newton-Raphson step (r <- r + r (1 - L r)), which squares the FP32
// estimate's relative error to ~2^-45; an exact division where Lf lies
// outside [2^-100, 2^100].
__device__ __forceinline__ double recip(double L, float Lf) {
  if (!(Lf > 0x1p-100f && Lf < 0x1p100f)) return 1.0 / L;
  const double r0 = widen(__frcp_rn(Lf));
  return fma(r0, fma(-L, r0, 1.0), r0);
}

// B[k] = beta T_k(tau), k < kDrMaxK (Chebyshev polynomials of the first kind).
__device__ __forceinline__ void chebyshev(double tau, double beta, double (&Bk)[kDrMaxK]) {
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
    Bk[k] = beta * T;
  }
}

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
  __shared__ double sg[kDrMaxK];
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
    a.tabs[c] = (a1 >= a0) ? fmax(fabs(a0), fabs(a1)) : 0.0;  // max |t| (0 with no finite time)
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
  const double df = (a.nfreq > 1) ? (a.freqs[a.nfreq - 1] - a.freqs[0]) / (double)(a.nfreq - 1) : 0.0;
  for (int64_t i = tid; i < n; i += blockDim.x) {
    DriftObs* const pay = reinterpret_cast<DriftObs*>(a.payload) + (o0 + i);
    double w = 0.0, x = 0.0;
    if (!cbad) {
      const double s = a.sigma[o0 + i];
      w = 1.0 / (s * s);
      x = a.x[o0 + i];
    }
    const double tau = (span > 0.0) ? 2.0 * (a.t[o0 + i] - lo) / span - 1.0 : 0.0;
    double Bk[kDrMaxK];
    chebyshev(tau, a.beta, Bk);
    float wb[kDrMaxK];
#pragma unroll
    for (int k = 0; k < kDrMaxK; ++k) {
      wb[k] = k < K ? (float)(w * Bk[k]) : 0.f;
      if (k < K) {
#pragma unroll
        for (int l = 0; l < kDrMaxK; ++l)
          if (l < K) acc[k * kDrMaxK + l] += w * Bk[k] * Bk[l];
        acc[kDrMaxK * kDrMaxK + k] += w * Bk[k] * x;
      }
    }
    DriftObs ob;
    ob.q = make_float4((float)(w * x), (float)w, wb[1], wb[2]);
    ob.D = isfinite(a.t[o0 + i]) ? phase_fixed64(a.t[o0 + i], df) : 0ull;
    ob.q3 = wb[3];
    ob.pad = 0.f;
    *pay = ob;
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
    for (int k = 0; k < kDrMaxK; ++k) sg[k] = g[k];
  }
  __syncthreads();
  // The bins sum w (x - B g), the residuals of the curve's baseline fit: their
  // bin sums are z_m = Y_m - Q_m . g itself, so a drift far above the noise
  // does not cancel inside FP32 sums of w x.
  if (K > 0 && !cbad)
    for (int64_t i = tid; i < n; i += blockDim.x) {
      const double s = a.sigma[o0 + i];
      const double tau = (span > 0.0) ? 2.0 * (a.t[o0 + i] - lo) / span - 1.0 : 0.0;
      double Bk[kDrMaxK];
      chebyshev(tau, a.beta, Bk);
      double r = a.x[o0 + i];
#pragma unroll
      for (int k = 0; k < kDrMaxK; ++k)
        if (k < K) r -= Bk[k] * sg[k];
      reinterpret_cast<DriftObs*>(a.payload)[o0 + i].q.x = (float)(r / (s * s));
    }
  if (blockIdx.x == 0)
    for (int64_t q = tid; q < a.nfreq; q += blockDim.x)
      if (!isfinite(a.freqs[q])) atomicOr(a.status, kStatusGrid);
}

// The binary64 reduction of one frequency from its bins (slots slot0 + m T):
// S = sum z^2 / L + v^T H^-1 v, H kept as its lower triangle. The constant
// basis function B_0 = beta has Q_m0 = beta Bw_m, and sum_i w_i B_ip =
// sum_m Q_mp, so its row of H and its entry of v take closed forms in the bin
// sums,
//   H_00 = 1 + beta^2 (1/alpha^2) sum_m Bw_m / L_m,
//   H_p0 = beta (1/alpha^2) sum_m Q_mp / L_m   (p >= 1),
//   v_0  = beta sum_m Bw_m z_m / L_m,
// (1 and 0 when 1/alpha^2 = 0) instead of H0 minus sums that cancel it.
template <int K>
__device__ __forceinline__ double drift_reduce(const DriftArgs& a, const unsigned char* bins, const float* bQ3,
                                               int slot0, int T, int64_t c) {
  constexpr bool kWide = K >= 2;
  const int M = a.M;
  double H[kDrMaxK][kDrMaxK], v[kDrMaxK];
  const double* h0 = a.H0 + c * kDrMaxK * kDrMaxK;
#pragma unroll
  for (int p = 0; p < K; ++p) {
    v[p] = 0.0;
#pragma unroll
    for (int q = 0; q <= p; ++q) H[p][q] = q == 0 ? 0.0 : h0[p * kDrMaxK + q];  // column 0: sums of 1/L terms
  }
  const double cal = a.inv_alpha2, beta = a.beta;
  const float calf = (float)cal;
  const bool finite_alpha = cal != 0.0;
  double S = 0.0;
  for (int m = 0; m < M; ++m) {
    const int sl = slot0 + m * T;
    double Y, Bw, Q[kDrMaxK];
    float bwf;
    if (kWide) {
      const float4 b = reinterpret_cast<const float4*>(bins)[sl];
      Y = widen(b.x);
      bwf = b.y;
      Q[1] = widen(b.z);
      if (K > 2) Q[2] = widen(b.w);
    } else {
      const float2 b = reinterpret_cast<const float2*>(bins)[sl];
      Y = widen(b.x);
      bwf = b.y;
    }
    Bw = widen(bwf);
    if (K > 3) Q[3] = widen(bQ3[sl]);
    const double L = Bw + cal;
    if (!(L > 0.0)) continue;  // empty bin with 1/alpha^2 = 0: dropped
    const double rL = recip(L, bwf + calf);
    const double z = Y;  // the bin's sum of w (x - B g)
    const double zl = z * rL;
    S += z * zl;
    if (K > 0) {
      v[0] += Bw * zl;
      if (finite_alpha) H[0][0] += Bw * rL;
    }
#pragma unroll
    for (int p = 1; p < K; ++p) {
      v[p] += Q[p] * zl;
      const double qs = Q[p] * rL;
      if (finite_alpha) H[p][0] += qs;
#pragma unroll
      for (int q = 1; q <= p; ++q) H[p][q] -= qs * Q[q];
    }
  }
  if (K > 0) {
    v[0] *= beta;
    H[0][0] = 1.0 + beta * beta * cal * H[0][0];
#pragma unroll
    for (int p = 1; p < K; ++p) H[p][0] *= beta * cal;
  }
  // v^T H^-1 v by Cholesky (H >= I): off-diagonal factors and the forward
  // substitution multiply by the reciprocal square roots of the pivots
  double Lc[kDrMaxK][kDrMaxK], di[kDrMaxK], y[kDrMaxK];
#pragma unroll
  for (int p = 0; p < K; ++p)
#pragma unroll
    for (int q = 0; q <= p; ++q) {
      double s = H[p][q];
#pragma unroll
      for (int r = 0; r < q; ++r) s -= Lc[p][r] * Lc[q][r];
      if (p == q)
        di[p] = s > 0.0 ? rsqrt(s) : 0.0;
      else
        Lc[p][q] = s * di[q];
    }
#pragma unroll
  for (int p = 0; p < K; ++p) {
    double s = v[p];
#pragma unroll
    for (int r = 0; r < p; ++r) s -= Lc[p][r] * y[r];
    y[p] = s * di[p];
    S += y[p] * y[p];
  }
  return S;
}

// One block per (tile of T frequencies, curve); thread = frequency. Bins
// thread-private (bank = lane), [M][T] slots of drift_bin_bytes(K): one packed
// read-modify-write per evaluation for K <= 3 (two for K = 4), two
// observations per iteration with all loads issued before the stores.
template <int K>
__global__ void __launch_bounds__(128) drift_kernel(const DriftArgs a) {
  constexpr bool kWide = K >= 2;  // (Y, Bw, Q_1, Q_2) as float4, else (Y, Bw) as float2
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, tid = threadIdx.x;
  const int M = a.M;
  const int64_t c = blockIdx.y, F = a.nfreq;
  const int64_t f0 = (int64_t)blockIdx.x * T, k = f0 + tid;
  unsigned char* const bins = smem;                                                     // [M][T] main slots
  float* const bQ3 = reinterpret_cast<float*>(bins + (size_t)M * T * (kWide ? 16 : 8));  // [M][T] (K = 4)
  ulonglong2* const sPD = reinterpret_cast<ulonglong2*>(smem + (size_t)M * T * drift_bin_bytes(K));  // [chunk]
  float4* const sQ = reinterpret_cast<float4*>(sPD + kDrChunk);                         // [chunk]
  float* const sQ3 = reinterpret_cast<float*>(sQ + kDrChunk);                           // [chunk] (K = 4)
  const bool grid_bad = (*(volatile unsigned*)a.status & kStatusGrid) != 0u;
  if (grid_bad) return;
  const bool cbad = a.curve_bad[c] != 0;
  const int64_t o0 = a.offsets[c], n = a.offsets[c + 1] - o0;
  const double df = (F > 1) ? (a.freqs[F - 1] - a.freqs[0]) / (double)(F - 1) : 0.0;
  const double fa = a.freqs[f0];
  // linear grid over this tile (the tile kernels' bound on the phase error)?
  const double tm = a.tabs[c];
  const double fk = k < F ? a.freqs[k] : fa;
  const bool nonlin = k < F && fabs(fk - fma((double)tid, df, fa)) * tm > kGridTolCycles;
  const bool lin = !__syncthreads_or(nonlin);
  for (int m = 0; m < M; ++m) {
    if (kWide)
      reinterpret_cast<float4*>(bins)[m * T + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    else
      reinterpret_cast<float2*>(bins)[m * T + tid] = make_float2(0.f, 0.f);
    if (K > 3) bQ3[m * T + tid] = 0.f;
  }
  const DriftObs* const obs = reinterpret_cast<const DriftObs*>(a.payload) + o0;
  for (int64_t oc = 0; oc < n; oc += kDrChunk) {
    const int cnt = (int)((n - oc) < kDrChunk ? (n - oc) : kDrChunk);
    __syncthreads();
    for (int i = tid; i < cnt; i += T) {
      const double ti = a.t[o0 + oc + i];
      const DriftObs ob = obs[oc + i];
      sPD[i] = lin ? make_ulonglong2(phase_fixed64(ti, fa), ob.D)
                   : make_ulonglong2((unsigned long long)__double_as_longlong(ti), 0ull);
      sQ[i] = ob.q;
      if (K > 3) sQ3[i] = ob.q3;
    }
    __syncthreads();
    if (!cbad) {
      auto slot = [&](const ulonglong2 pd) {
        const unsigned long long phi =
            lin ? pd.x + (unsigned long long)tid * pd.y : phase_fixed64(__longlong_as_double((long long)pd.x), fk);
        return (int)bin_of_phase(phi, (unsigned)M) * T + tid;
      };
      // two observations per iteration: both read-modify-write chains are in
      // flight at once; where both fall in one bin the second update starts
      // from the first one's sum (same additions in the same order)
      int i = 0;
      for (; i + 1 < cnt; i += 2) {
        const int ma = slot(sPD[i]), mb = slot(sPD[i + 1]);
        const float4 pa = sQ[i], pb = sQ[i + 1];
        if (kWide) {
          float4* const b4 = reinterpret_cast<float4*>(bins);
          const float4 va = b4[ma];
          float4 vb = b4[mb];
          const float4 ua = make_float4(va.x + pa.x, va.y + pa.y, va.z + pa.z, va.w + pa.w);
          if (ma == mb) vb = ua;
          b4[ma] = ua;
          b4[mb] = make_float4(vb.x + pb.x, vb.y + pb.y, vb.z + pb.z, vb.w + pb.w);
        } else {
          float2* const b2 = reinterpret_cast<float2*>(bins);
          const float2 va = b2[ma];
          float2 vb = b2[mb];
          const float2 ua = make_float2(va.x + pa.x, va.y + pa.y);
          if (ma == mb) vb = ua;
          b2[ma] = ua;
          b2[mb] = make_float2(vb.x + pb.x, vb.y + pb.y);
        }
        if (K > 3) {
          const float qa = bQ3[ma];
          float qb = bQ3[mb];
          const float ra = qa + sQ3[i];
          if (ma == mb) qb = ra;
          bQ3[ma] = ra;
          bQ3[mb] = qb + sQ3[i + 1];
        }
      }
      if (i < cnt) {
        const int ma = slot(sPD[i]);
        const float4 pa = sQ[i];
        if (kWide) {
          float4* const b4 = reinterpret_cast<float4*>(bins);
          const float4 va = b4[ma];
          b4[ma] = make_float4(va.x + pa.x, va.y + pa.y, va.z + pa.z, va.w + pa.w);
        } else {
          float2* const b2 = reinterpret_cast<float2*>(bins);
          const float2 va = b2[ma];
          b2[ma] = make_float2(va.x + pa.x, va.y + pa.y);
        }
        if (K > 3) bQ3[ma] += sQ3[i];
      }
    }
  }
  if (k >= F) return;
  const double S = drift_reduce<K>(a, bins, bQ3, tid, T, c);
  const float Sf = cbad ? __int_as_float(0x7fc00000) : (float)S;
  if (a.S32) a.S32[c * F + k] = Sf;
  if (a.S_out) a.S_out[c * F + k] = cbad ? (double)Sf : S;
}

// As drift_kernel, with R consecutive frequencies per thread: tiles of T R
// frequencies, [r][M][T] bin slots, each staged observation serving the
// thread's R frequencies (half the broadcast per evaluation for R = 2, twice
// the bins per thread). A separate kernel: the one-frequency loop above runs
// faster in its own form.
template <int K, int R>
__global__ void __launch_bounds__(128) drift_kernel_rf(const DriftArgs a) {
  constexpr bool kWide = K >= 2;  // (Y, Bw, Q_1, Q_2) as float4, else (Y, Bw) as float2
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, tid = threadIdx.x;
  const int M = a.M, MT = M * T;
  const int64_t c = blockIdx.y, F = a.nfreq;
  const int64_t f0 = (int64_t)blockIdx.x * (T * R);
  const int j0 = tid * R;  // the thread's first frequency within the tile
  unsigned char* const bins = smem;                                                         // [R][M][T] main slots
  float* const bQ3 = reinterpret_cast<float*>(bins + (size_t)R * MT * (kWide ? 16 : 8));    // [R][M][T] (K = 4)
  ulonglong2* const sPD = reinterpret_cast<ulonglong2*>(smem + (size_t)R * MT * drift_bin_bytes(K));  // [chunk]
  float4* const sQ = reinterpret_cast<float4*>(sPD + kDrChunk);                             // [chunk]
  float* const sQ3 = reinterpret_cast<float*>(sQ + kDrChunk);                               // [chunk] (K = 4)
  const bool grid_bad = (*(volatile unsigned*)a.status & kStatusGrid) != 0u;
  if (grid_bad) return;
  const bool cbad = a.curve_bad[c] != 0;
  const int64_t o0 = a.offsets[c], n = a.offsets[c + 1] - o0;
  const double df = (F > 1) ? (a.freqs[F - 1] - a.freqs[0]) / (double)(F - 1) : 0.0;
  const double fa = a.freqs[f0];
  // linear grid over this tile (the tile kernels' bound on the phase error)?
  const double tm = a.tabs[c];
  double fk[R];
  bool nonlin = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t k = f0 + j0 + r;
    fk[r] = k < F ? a.freqs[k] : fa;
    if (k < F && fabs(fk[r] - fma((double)(j0 + r), df, fa)) * tm > kGridTolCycles) nonlin = true;
  }
  const bool lin = !__syncthreads_or(nonlin);
  for (int q = 0; q < R * M; ++q) {
    if (kWide)
      reinterpret_cast<float4*>(bins)[q * T + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    else
      reinterpret_cast<float2*>(bins)[q * T + tid] = make_float2(0.f, 0.f);
    if (K > 3) bQ3[q * T + tid] = 0.f;
  }
  const DriftObs* const obs = reinterpret_cast<const DriftObs*>(a.payload) + o0;
  for (int64_t oc = 0; oc < n; oc += kDrChunk) {
    const int cnt = (int)((n - oc) < kDrChunk ? (n - oc) : kDrChunk);
    __syncthreads();
    for (int i = tid; i < cnt; i += T) {
      const double ti = a.t[o0 + oc + i];
      const DriftObs ob = obs[oc + i];
      sPD[i] = lin ? make_ulonglong2(phase_fixed64(ti, fa), ob.D)
                   : make_ulonglong2((unsigned long long)__double_as_longlong(ti), 0ull);
      sQ[i] = ob.q;
      if (K > 3) sQ3[i] = ob.q3;
    }
    __syncthreads();
    if (!cbad) {
      // the observation's slot for each of the thread's R frequencies
      auto slots = [&](const ulonglong2 pd, int (&sl)[R]) {
        if (lin) {
          unsigned long long phi = pd.x + (unsigned long long)j0 * pd.y;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            sl[r] = r * MT + (int)bin_of_phase(phi, (unsigned)M) * T + tid;
            phi += pd.y;
          }
        } else {
          const double ti = __longlong_as_double((long long)pd.x);
#pragma unroll
          for (int r = 0; r < R; ++r) sl[r] = r * MT + (int)bin_of_phase(phase_fixed64(ti, fk[r]), (unsigned)M) * T + tid;
        }
      };
      // two observations per iteration: all read-modify-write chains are in
      // flight at once; where both observations fall in one bin the second
      // update starts from the first one's sum (same additions in the same order)
      int i = 0;
      for (; i + 1 < cnt; i += 2) {
        int sa[R], sb[R];
        slots(sPD[i], sa);
        slots(sPD[i + 1], sb);
        const float4 pa = sQ[i], pb = sQ[i + 1];
        if (kWide) {
          float4* const b4 = reinterpret_cast<float4*>(bins);
          float4 va[R], vb[R];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            va[r] = b4[sa[r]];
            vb[r] = b4[sb[r]];
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float4 ua = make_float4(va[r].x + pa.x, va[r].y + pa.y, va[r].z + pa.z, va[r].w + pa.w);
            const float4 wb = sa[r] == sb[r] ? ua : vb[r];
            b4[sa[r]] = ua;
            b4[sb[r]] = make_float4(wb.x + pb.x, wb.y + pb.y, wb.z + pb.z, wb.w + pb.w);
          }
        } else {
          float2* const b2 = reinterpret_cast<float2*>(bins);
          float2 va[R], vb[R];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            va[r] = b2[sa[r]];
            vb[r] = b2[sb[r]];
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float2 ua = make_float2(va[r].x + pa.x, va[r].y + pa.y);
            const float2 wb = sa[r] == sb[r] ? ua : vb[r];
            b2[sa[r]] = ua;
            b2[sb[r]] = make_float2(wb.x + pb.x, wb.y + pb.y);
          }
        }
        if (K > 3) {
          const float ra = sQ3[i], rb = sQ3[i + 1];
          float qa[R], qb[R];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            qa[r] = bQ3[sa[r]];
            qb[r] = bQ3[sb[r]];
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float ua = qa[r] + ra;
            bQ3[sa[r]] = ua;
            bQ3[sb[r]] = (sa[r] == sb[r] ? ua : qb[r]) + rb;
          }
        }
      }
      if (i < cnt) {
        int sa[R];
        slots(sPD[i], sa);
        const float4 pa = sQ[i];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (kWide) {
            float4* const b4 = reinterpret_cast<float4*>(bins);
            const float4 va = b4[sa[r]];
            b4[sa[r]] = make_float4(va.x + pa.x, va.y + pa.y, va.z + pa.z, va.w + pa.w);
          } else {
            float2* const b2 = reinterpret_cast<float2*>(bins);
            const float2 va = b2[sa[r]];
            b2[sa[r]] = make_float2(va.x + pa.x, va.y + pa.y);
          }
          if (K > 3) bQ3[sa[r]] += sQ3[i];
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t k = f0 + j0 + r;
    if (k >= F) break;
    const double S = drift_reduce<K>(a, bins, bQ3, r * MT + tid, T, c);
    const float Sf = cbad ? __int_as_float(0x7fc00000) : (float)S;
    if (a.S32) a.S32[c * F + k] = Sf;
    if (a.S_out) a.S_out[c * F + k] = cbad ? (double)Sf : S;
  }
}

const void* drift_fn(int K, int R) {
  if (R == 2) {
    switch (K) {
      case 0: return reinterpret_cast<const void*>(&drift_kernel_rf<0, 2>);
      case 1: return reinterpret_cast<const void*>(&drift_kernel_rf<1, 2>);
      case 2: return reinterpret_cast<const void*>(&drift_kernel_rf<2, 2>);
      case 3: return reinterpret_cast<const void*>(&drift_kernel_rf<3, 2>);
      default: return reinterpret_cast<const void*>(&drift_kernel_rf<4, 2>);
    }
  }
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
  if (cudaFuncGetAttributes(&fa, drift_fn(4, 2)) != cudaSuccess) return 0;
  return smem_optin > (int)fa.sharedSizeBytes ? (size_t)(smem_optin - (int)fa.sharedSizeBytes) : 0;
}

int drift_threads(int M, int K, int smem_optin) {
  const size_t lim = drift_dynamic_limit(smem_optin);
  for (int T = 128; T >= 32; T >>= 1)
    if (drift_smem_bytes(M, K, T, 1) <= lim) return T;
  return 0;
}

bool drift_fits(int M, int K, int T, int R, int smem_optin) {
  return drift_smem_bytes(M, K, T, R) <= drift_dynamic_limit(smem_optin);
}

size_t drift_smem_bytes(int M, int K, int T, int R) {
  return (size_t)R * M * T * drift_bin_bytes(K) + (size_t)kDrChunk * drift_stage_bytes(K);
}

int drift_max_basis() { return kDrMaxK; }

size_t drift_payload_bytes() { return sizeof(DriftObs); }

cudaError_t drift_init_attributes(int max_smem) {
  const int lim = (int)drift_dynamic_limit(max_smem);
  for (int K = 0; K <= kDrMaxK; ++K)
    for (int R = 1; R <= 2; ++R) {
      const cudaError_t e = cudaFuncSetAttribute(drift_fn(K, R), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

cudaError_t launch_drift(const DriftArgs& a, int T, int R, cudaStream_t st) {
  if (a.ncurves <= 0) return cudaSuccess;
  drift_prep_kernel<<<(unsigned)a.ncurves, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.nfreq <= 0) return e;
  const int64_t tiles = (a.nfreq + (int64_t)T * R - 1) / ((int64_t)T * R);
  if (a.timing_start) cudaEventRecord(a.timing_start, st);
  void* params[] = {const_cast<DriftArgs*>(&a)};
  e = cudaLaunchKernel(drift_fn(a.K, R), dim3((unsigned)tiles, (unsigned)a.ncurves), dim3(T), params,
                       drift_smem_bytes(a.M, a.K, T, R), st);
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
