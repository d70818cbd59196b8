// Persistent FPW tile kernel: Eq. 1 (Section 2) for every (curve, frequency)
// of a work list, with the per-curve top-k peaks of Section 3.5.
//
// Work decomposition
//   A work item is (curve c, frequency segment [f_lo, f_hi)). Thread blocks pop
//   items from a global counter (items are sorted by cost, longest first).
//   Within an item the segment is swept in tiles of W = T * R consecutive
//   frequencies: thread j owns frequencies s + j*R + r (r < R). Tiles overlap by
//   two frequencies so that every owned frequency has both neighbours in the
//   same tile (needed for the local-maximum test of the peak finder).
//
// Per tile
//   1. Anchor: for each observation, Phi_s = frac(t_i * f_s) as a 64-bit
//      fixed-point fraction from the exact integer product of the binary64
//      significands, and the step D_i = frac(t_i * df) (df = grid spacing).
//      Both are staged in shared memory with a_i = x_i w_i and w_i (prep output).
//   2. Hot loop (per observation, per thread, per r): Phi = Phi_s + (j*R + r) D_i
//      (mod 2^64), bin m = floor(M * Phi_hi / 2^32), A_m += a_i, B_m += w_i in a
//      thread-private [r][m][thread] bin array in shared memory (bank = lane, so
//      conflict-free), all R loads issued before the R stores.
//   3. Reduce: S = sum_m A_m^2 / (B_m + 1/alpha^2), empty bins contribute 0.
//   4. Peaks: local maxima among owned frequencies, merged into the item's
//      running top-k (shared memory), written as candidates at the item's end.
//
// Grids that are not linear to within kGridTolCycles over a tile fall back to a
// direct exact anchor per (observation, frequency).
#include <math.h>

#include "fpw_internal.cuh"

namespace fpw {
namespace {

template <typename A>
struct Acc2;
template <>
struct Acc2<float> {
  using T = float2;
};
template <>
struct Acc2<double> {
  using T = double2;
};

__device__ __forceinline__ float2 acc_add(float2 a, float2 b) { return f2add(a, b); }
__device__ __forceinline__ double2 acc_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ void acc_zero(float2& v) { v = make_float2(0.f, 0.f); }
__device__ __forceinline__ void acc_zero(double2& v) { v = make_double2(0.0, 0.0); }

// n / d for the reduce step: the fast reciprocal-based quotient (2 ulp) in the
// normal range of d, correctly rounded division elsewhere; binary64 always
// correctly rounded.
__device__ __forceinline__ float quotient(float n, float d) {
  return (d >= 1.17549435e-38f && d <= 8.5e37f) ? __fdividef(n, d) : n / d;
}
__device__ __forceinline__ double quotient(double n, double d) { return n / d; }

struct Layout {
  size_t bins, pd, aw, candS, candI, topS, topI, edges, red, misc, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline Layout tile_layout(int T, int R, int M, int NC, bool acc64) {
  const size_t a2 = acc64 ? 16 : 8;
  const size_t W = (size_t)T * R;
  Layout L;
  size_t o = 0;
  L.bins = o;
  o = align16(o + (size_t)R * M * T * a2);
  L.pd = o;
  o = align16(o + (size_t)NC * 16);
  L.aw = o;
  o = align16(o + (size_t)NC * a2);
  L.candS = o;
  o = align16(o + W * 8);
  L.candI = o;
  o = align16(o + W * 4);
  L.topS = o;
  o = align16(o + (size_t)FPW_MAX_TOPK * 8);
  L.topI = o;
  o = align16(o + (size_t)FPW_MAX_TOPK * 4);
  L.edges = o;
  o = align16(o + (size_t)(T / 32) * 2 * 8);
  L.red = o;
  o = align16(o + 32 * 8);
  L.misc = o;
  o = align16(o + 64);
  L.total = o;
  return L;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Selects the best kk entries of (top list) + (candidate list) into the top
// list, ranked by S descending then index ascending. Executed by one warp.
// Entries with index < 0 are empty. kk <= FPW_MAX_TOPK (two results per lane).
__device__ void warp_merge_topk(double* topS, int* topI, int kk, double* cS, int* cI, int cnt, int lane) {
  double keepS[2] = {-INFINITY, -INFINITY};
  int keepI[2] = {-1, -1};
  const int pool = kk + cnt;
  for (int q = 0; q < kk; ++q) {
    double bs = -INFINITY;
    int bi = -1, bp = -1;
    for (int e = lane; e < pool; e += 32) {
      const double s = (e < kk) ? topS[e] : cS[e - kk];
      const int i = (e < kk) ? topI[e] : cI[e - kk];
      if (i >= 0 && (bp < 0 || ranks_before(s, i, bs, bi))) {
        bs = s;
        bi = i;
        bp = e;
      }
    }
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
    if (lane == 0 && bp >= 0) {
      if (bp < kk)
        topI[bp] = -1;
      else
        cI[bp - kk] = -1;
    }
    if (lane == (q & 31)) {
      keepS[q >> 5] = (bp >= 0) ? bs : -INFINITY;
      keepI[q >> 5] = (bp >= 0) ? bi : -1;
    }
    __syncwarp();
  }
  for (int q = lane; q < kk; q += 32) {
    topS[q] = keepS[q >> 5];
    topI[q] = keepI[q >> 5];
  }
  __syncwarp();
}

template <int R, int PHASE, typename A>
__global__ void __launch_bounds__(512) tile_kernel(const TileArgs args) {
  using A2 = typename Acc2<A>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
  const int M = args.M, NC = args.obs_chunk, kk = args.k;
  const Layout L = tile_layout(T, R, M, NC, sizeof(A) == 8);
  unsigned char* const my_bins = smem + L.bins + (size_t)tid * sizeof(A2);
  ulonglong2* const sPD = reinterpret_cast<ulonglong2*>(smem + L.pd);
  A2* const sAW = reinterpret_cast<A2*>(smem + L.aw);
  double* const candS = reinterpret_cast<double*>(smem + L.candS);
  int* const candI = reinterpret_cast<int*>(smem + L.candI);
  double* const topS = reinterpret_cast<double*>(smem + L.topS);
  int* const topI = reinterpret_cast<int*>(smem + L.topI);
  double* const edges = reinterpret_cast<double*>(smem + L.edges);
  double* const red = reinterpret_cast<double*>(smem + L.red);
  int* const misc = reinterpret_cast<int*>(smem + L.misc);

  const int64_t F = args.nfreq;
  const int W = T * R;
  const unsigned T8 = (unsigned)T * (unsigned)sizeof(A2);
  const unsigned MT8 = (unsigned)M * T8;
  const double df = (F > 1) ? (args.freqs[F - 1] - args.freqs[0]) / (double)(F - 1) : 0.0;
  const bool grid_bad = (*(volatile unsigned*)args.status & kStatusGrid) != 0u;
  const A cal = (A)args.inv_alpha2;
  const unsigned j0 = (unsigned)tid * R;

  // bins start at zero; every reduce leaves them zero again
  for (int q = 0; q < R * M; ++q) {
    A2 z;
    acc_zero(z);
    *reinterpret_cast<A2*>(my_bins + (size_t)q * T8) = z;
  }

  for (;;) {
    if (tid == 0) misc[0] = (int)atomicAdd(args.counter, 1u);
    __syncthreads();
    const int it = misc[0];
    if (it >= args.nitems) break;
    const WorkItem wi = args.items[it];
    const int c = wi.curve;
    int64_t base = 0, n = args.n_single;
    if (args.offsets) {
      base = args.offsets[c];
      n = args.offsets[c + 1] - base;
    }
    if (grid_bad || args.curve_bad[c]) {
      if (args.S_out)
        for (int64_t q = wi.f_lo + tid; q < wi.f_hi; q += T) args.S_out[(int64_t)c * F + q] = __longlong_as_double(0x7ff8000000000000ll);
      if (kk > 0)
        for (int q = tid; q < kk; q += T) {
          args.cand_S[(int64_t)wi.slot * kk + q] = -INFINITY;
          args.cand_idx[(int64_t)wi.slot * kk + q] = -1;
        }
      __syncthreads();
      continue;
    }
    // largest |t| of the curve (sets the grid-linearity tolerance)
    double tm = 0.0;
    for (int64_t i = tid; i < n; i += T) tm = fmax(tm, fabs(args.t[base + i]));
    tm = warp_max(tm);
    if (lane == 0) red[warp] = tm;
    for (int q = tid; q < kk; q += T) {
      topS[q] = -INFINITY;
      topI[q] = -1;
    }
    if (tid == 0) misc[1] = 0;
    __syncthreads();
    tm = 0.0;
    for (int w = 0; w < nwarps; ++w) tm = fmax(tm, red[w]);
    const bool resident = n <= NC;
    bool staged_lin = false;

    for (int64_t s = (int64_t)wi.f_lo - 1; s + 1 < wi.f_hi; s += W - 2) {
      const int64_t a = s < 0 ? 0 : s;
      const double fa = args.freqs[a];
      // grid linearity over this tile: the precomputed per-tile deviation when
      // available (tile starts sit at multiples of W-2, minus one), else checked here
      bool lin;
      if (args.tile_dev) {
        lin = args.tile_dev[(s + 1) / (W - 2)] * tm <= kGridTolCycles;
      } else {
        bool nonlin = false;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int64_t k = s + (int64_t)j0 + r;
          if (k >= 0 && k < F) {
            const double pred = fma((double)(k - a), df, fa);
            if (fabs(args.freqs[k] - pred) * tm > kGridTolCycles) nonlin = true;
          }
        }
        lin = !__syncthreads_or(nonlin);
      }
      // a curve that fits in one chunk keeps D_i and (a_i, w_i) staged across the
      // tiles of an item; only the anchor phase is recomputed per tile
      const bool keep = resident && staged_lin && lin;

      for (int64_t o = 0; o < n; o += NC) {
        const int cnt = (int)((n - o) < NC ? (n - o) : NC);
        for (int i = tid; i < cnt; i += T) {
          const double ti = args.t[base + o + i];
          if (keep) {
            const unsigned long long D = sPD[i].y;
            unsigned long long P = phase_fixed64(ti, fa);
            if (s < a) P -= D;  // tile starts one step before frequency 0
            sPD[i].x = P;
          } else {
            ulonglong2 pd;
            if (lin) {
              const unsigned long long D = phase_fixed64(ti, df);
              unsigned long long P = phase_fixed64(ti, fa);
              if (s < a) P -= D;
              pd = make_ulonglong2(P, D);
            } else {
              pd = make_ulonglong2((unsigned long long)__double_as_longlong(ti), 0ull);
            }
            sPD[i] = pd;
            sAW[i] = reinterpret_cast<const A2*>(args.aw)[base + o + i];
          }
        }
        staged_lin = lin;
        __syncthreads();
        if (lin && PHASE == FPW_PHASE_FIXED64) {
          // The next observation's staged data is loaded before this one's bin
          // stores (the compiler cannot move it there itself: both are shared
          // memory), so the broadcast-load latency overlaps the bin updates.
          ulonglong2 pd = sPD[0];
          A2 aw = sAW[0];
#pragma unroll 2
          for (int i = 0; i < cnt; ++i) {
            const int in = (i + 1 < cnt) ? i + 1 : i;
            const ulonglong2 pdn = sPD[in];
            const A2 awn = sAW[in];
            unsigned long long phi = pd.x + (unsigned long long)j0 * pd.y;
            unsigned off[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              off[r] = bin_of_phase(phi, (unsigned)M) * T8 + (unsigned)r * MT8;
              phi += pd.y;
            }
            A2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = *reinterpret_cast<const A2*>(my_bins + off[r]);
#pragma unroll
            for (int r = 0; r < R; ++r) *reinterpret_cast<A2*>(my_bins + off[r]) = acc_add(v[r], aw);
            pd = pdn;
            aw = awn;
          }
        } else if (lin) {  // FPW_PHASE_FP32: FP32 phase from an FP32 anchor every K frequencies
          const int K = args.K;
          float jr[R];
          long long da[R];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const long long k = s + (long long)j0 + r;
            const long long ak = (k >= 0) ? k - (k % K) : 0;
            jr[r] = (float)(k - ak);
            da[r] = ak - s;
          }
          for (int i = 0; i < cnt; ++i) {
            const ulonglong2 pd = sPD[i];
            const A2 aw = sAW[i];
            const float d32 = (float)(unsigned)(pd.y >> 32) * 0x1p-32f;
            unsigned off[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const unsigned long long pa = pd.x + (unsigned long long)da[r] * pd.y;
              const float p32 = (float)(unsigned)(pa >> 32) * 0x1p-32f;
              float p = fmaf(jr[r], d32, p32);
              p = p - floorf(p);
              unsigned m = (unsigned)(p * (float)M);
              m = m < (unsigned)M ? m : (unsigned)M - 1u;
              off[r] = m * T8 + (unsigned)r * MT8;
            }
            A2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = *reinterpret_cast<const A2*>(my_bins + off[r]);
#pragma unroll
            for (int r = 0; r < R; ++r) *reinterpret_cast<A2*>(my_bins + off[r]) = acc_add(v[r], aw);
          }
        } else {  // non-linear grid: exact anchor per (observation, frequency)
          double fr[R];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            int64_t k = s + (int64_t)j0 + r;
            k = k < 0 ? 0 : (k >= F ? F - 1 : k);
            fr[r] = args.freqs[k];
          }
          for (int i = 0; i < cnt; ++i) {
            const double ti = __longlong_as_double((long long)sPD[i].x);
            const A2 aw = sAW[i];
            unsigned off[R];
#pragma unroll
            for (int r = 0; r < R; ++r) off[r] = bin_of_phase(phase_fixed64(ti, fr[r]), (unsigned)M) * T8 + (unsigned)r * MT8;
            A2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = *reinterpret_cast<const A2*>(my_bins + off[r]);
#pragma unroll
            for (int r = 0; r < R; ++r) *reinterpret_cast<A2*>(my_bins + off[r]) = acc_add(v[r], aw);
          }
        }
        __syncthreads();
      }

      // reduce to S (and clear the bins for the next tile); S and the peak test
      // stay in the accumulation type (no binary64 work for FP32 sums)
      A S[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        A acc = (A)0;
        unsigned char* b = my_bins + (size_t)r * MT8;
        for (int m = 0; m < M; ++m) {
          A2* p = reinterpret_cast<A2*>(b + (size_t)m * T8);
          const A2 v = *p;
          A2 z;
          acc_zero(z);
          *p = z;
          const A den = v.y + cal;
          acc += (den > (A)0) ? quotient(v.x * v.x, den) : (A)0;
        }
        const int64_t k = s + (int64_t)j0 + r;
        S[r] = (k >= 0 && k < F) ? acc : (A)-INFINITY;
      }
      // dense output of owned frequencies
      if (args.S_out) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int j = (int)j0 + r;
          const int64_t k = s + j;
          if (j > 0 && j < W - 1 && k >= wi.f_lo && k < wi.f_hi) args.S_out[(int64_t)c * F + k] = (double)S[r];
        }
      }
      if (kk > 0) {
        // neighbours across lanes and warps
        A left = __shfl_up_sync(0xffffffffu, S[R - 1], 1);
        A right = __shfl_down_sync(0xffffffffu, S[0], 1);
        A* const aedges = reinterpret_cast<A*>(edges);
        if (lane == 0) aedges[2 * warp] = S[0];
        if (lane == 31) aedges[2 * warp + 1] = S[R - 1];
        __syncthreads();
        if (lane == 0) left = (warp > 0) ? aedges[2 * warp - 1] : (A)-INFINITY;
        if (lane == 31) right = (warp + 1 < nwarps) ? aedges[2 * warp + 2] : (A)-INFINITY;
        const A thr = (topI[kk - 1] >= 0) ? (A)topS[kk - 1] : (A)-INFINITY;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int j = (int)j0 + r;
          const int64_t k = s + j;
          const bool owned = j > 0 && j < W - 1 && k >= wi.f_lo && k < wi.f_hi;
          const A prev = (r > 0) ? S[r > 0 ? r - 1 : 0] : left;
          const A next = (r < R - 1) ? S[r < R - 1 ? r + 1 : 0] : right;
          const bool peak = args.peak_raw ? owned : (owned && S[r] > prev && S[r] >= next);
          if (peak && S[r] > thr) {
            const int slot = atomicAdd(&misc[1], 1);
            candS[slot] = (double)S[r];
            candI[slot] = (int)k;
          }
        }
        __syncthreads();
        const int cnt = misc[1];
        if (cnt > 0) {
          if (warp == 0) warp_merge_topk(topS, topI, kk, candS, candI, cnt, lane);
          __syncthreads();
          if (tid == 0) misc[1] = 0;
        }
      }
      __syncthreads();
    }
    if (kk > 0)
      for (int q = tid; q < kk; q += T) {
        args.cand_S[(int64_t)wi.slot * kk + q] = topS[q];
        args.cand_idx[(int64_t)wi.slot * kk + q] = topI[q];
      }
    __syncthreads();
  }
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
    d = warp_max(d);
    if (lane == 0) dev[q] = d;
  }
}

template <int R, int PHASE, typename A>
const void* tile_fn() {
  return reinterpret_cast<const void*>(&tile_kernel<R, PHASE, A>);
}

const void* pick(int R, int phase_mode, bool acc64) {
  const bool fp32p = phase_mode == FPW_PHASE_FP32;
#define FPW_PICK(RR)                                                                                  \
  if (R == RR) {                                                                                      \
    if (acc64) return fp32p ? tile_fn<RR, FPW_PHASE_FP32, double>() : tile_fn<RR, FPW_PHASE_FIXED64, double>(); \
    return fp32p ? tile_fn<RR, FPW_PHASE_FP32, float>() : tile_fn<RR, FPW_PHASE_FIXED64, float>();    \
  }
  FPW_PICK(1)
  FPW_PICK(2)
  FPW_PICK(4)
  FPW_PICK(8)
#undef FPW_PICK
  return nullptr;
}

}  // namespace

size_t tile_smem_bytes(int T, int R, int M, int NC, int /*k*/, bool accum64) {
  return tile_layout(T, R, M, NC, accum64).total;
}

bool tile_supported_R(int R) { return R == 1 || R == 2 || R == 4 || R == 8; }

cudaError_t tile_init_attributes(int max_smem) {
  for (int R : {1, 2, 4, 8})
    for (int ph : {FPW_PHASE_FIXED64, FPW_PHASE_FP32})
      for (int acc : {0, 1}) {
        cudaError_t e = cudaFuncSetAttribute(pick(R, ph, acc != 0), cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
      }
  return cudaSuccess;
}

int tile_max_blocks_per_sm(int R, int phase_mode, bool accum64, int T, size_t smem) {
  const void* fn = pick(R, phase_mode, accum64);
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

cudaError_t launch_tile(const TileArgs& a, const TileShape& s, int phase_mode, bool accum64, int grid,
                        cudaStream_t st) {
  const void* fn = pick(s.R, phase_mode, accum64);
  if (!fn) return cudaErrorInvalidValue;
  void* params[] = {const_cast<TileArgs*>(&a)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(s.threads), params, s.smem, st);
}

}  // namespace fpw
