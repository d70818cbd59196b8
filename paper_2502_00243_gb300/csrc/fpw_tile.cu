// Persistent FPW tile kernels: Eq. 1 (Section 2) for every (curve, frequency)
// of a work list, with the per-curve top-k peaks of Section 3.5; and the same
// with several bin counts M = M_max / g derived from one M_max pass (Section 3.4).
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
//      Several-M kernel: in-place prefix sums of the M_max bins, then for each
//      group g the windows of g consecutive bins (circularly) for every offset;
//      S_g(f) is the largest S over the g offsets, and that offset is kept.
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
__device__ __forceinline__ float2 acc_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
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

__host__ __device__ inline Layout tile_layout(int T, int R, int M, int NC, bool acc64, int ngroups) {
  const size_t a2 = acc64 ? 16 : 8;
  const size_t W = (size_t)T * R;
  const size_t tops = (size_t)(ngroups > 1 ? ngroups : 1) * FPW_MAX_TOPK;
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
  o = align16(o + tops * 8);
  L.topI = o;
  o = align16(o + tops * 4);
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
// list, ranked by S descending then key ascending. Executed by one warp.
// Entries with key < 0 are empty. kk <= FPW_MAX_TOPK (two results per lane).
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

// Per-block view of shared memory and the constants every stage needs.
template <typename A>
struct Block {
  using A2 = typename Acc2<A>::T;
  unsigned char* my_bins;  // this thread's column of the [r][m][thread] bin array
  ulonglong2* sPD;         // staged {Phi_s, D} per observation
  A2* sAW;                 // staged {a, w} per observation
  double* candS;
  int* candI;
  double* topS;            // [groups][FPW_MAX_TOPK]
  int* topI;
  double* edges;
  double* red;
  int* misc;
  int T, tid, lane, warp, nwarps, M, NC, kk, W;
  unsigned T8, MT8, j0;
  int64_t F;
  double df;
};

template <int R, typename A>
__device__ __forceinline__ Block<A> make_block(unsigned char* smem, const TileArgs& args) {
  using A2 = typename Acc2<A>::T;
  Block<A> b;
  b.T = blockDim.x;
  b.tid = threadIdx.x;
  b.lane = b.tid & 31;
  b.warp = b.tid >> 5;
  b.nwarps = b.T >> 5;
  b.M = args.M;
  b.NC = args.obs_chunk;
  b.kk = args.k;
  b.W = b.T * R;
  const Layout L = tile_layout(b.T, R, b.M, b.NC, sizeof(A) == 8, args.ngroups);
  b.my_bins = smem + L.bins + (size_t)b.tid * sizeof(A2);
  b.sPD = reinterpret_cast<ulonglong2*>(smem + L.pd);
  b.sAW = reinterpret_cast<A2*>(smem + L.aw);
  b.candS = reinterpret_cast<double*>(smem + L.candS);
  b.candI = reinterpret_cast<int*>(smem + L.candI);
  b.topS = reinterpret_cast<double*>(smem + L.topS);
  b.topI = reinterpret_cast<int*>(smem + L.topI);
  b.edges = reinterpret_cast<double*>(smem + L.edges);
  b.red = reinterpret_cast<double*>(smem + L.red);
  b.misc = reinterpret_cast<int*>(smem + L.misc);
  b.T8 = (unsigned)b.T * (unsigned)sizeof(A2);
  b.MT8 = (unsigned)b.M * b.T8;
  b.j0 = (unsigned)b.tid * R;
  b.F = args.nfreq;
  b.df = (b.F > 1) ? (args.freqs[b.F - 1] - args.freqs[0]) / (double)(b.F - 1) : 0.0;
  return b;
}

// Is the grid linear over the tile starting at s? The precomputed per-tile
// deviation when available (tile starts sit at multiples of W-2, minus one),
// else checked here (block-wide).
template <int R, typename A>
__device__ __forceinline__ bool tile_is_linear(const TileArgs& args, const Block<A>& b, int64_t s, int64_t a,
                                               double fa, double tm) {
  if (args.tile_dev) return args.tile_dev[(s + 1) / (b.W - 2)] * tm <= kGridTolCycles;
  bool nonlin = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t k = s + (int64_t)b.j0 + r;
    if (k >= 0 && k < b.F) {
      const double pred = fma((double)(k - a), b.df, fa);
      if (fabs(args.freqs[k] - pred) * tm > kGridTolCycles) nonlin = true;
    }
  }
  return !__syncthreads_or(nonlin);
}

// Stages every observation chunk of the curve for the tile starting at s and
// accumulates its bins (steps 1 and 2). A curve that fits in one chunk keeps
// D_i and (a_i, w_i) staged across the tiles of an item (keep); only the anchor
// phase is then recomputed.
template <int R, int PHASE, typename A>
__device__ __forceinline__ void accumulate_tile(const TileArgs& args, const Block<A>& b, int64_t s, int64_t a,
                                                double fa, bool lin, bool keep, bool& staged_lin, int64_t base,
                                                int64_t n) {
  using A2 = typename Acc2<A>::T;
  const int T = b.T, tid = b.tid, NC = b.NC;
  const unsigned M = (unsigned)b.M, T8 = b.T8, MT8 = b.MT8, j0 = b.j0;
  unsigned char* const my_bins = b.my_bins;
  ulonglong2* const sPD = b.sPD;
  A2* const sAW = b.sAW;
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
          const unsigned long long D = phase_fixed64(ti, b.df);
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
      if (R == 2) {
        // Software-pipelined (measured faster only at R = 2, where the phase ->
        // bin -> offset chain is a larger share of each iteration): the bin
        // offsets of observation i + 1 are computed while observation i's bin
        // loads are in flight, from staged data loaded one iteration earlier.
        // Same adds in the same order as the loop below.
        unsigned off[R];
        {
          const ulonglong2 p0 = sPD[0];
          const unsigned long long f0 = p0.x + (unsigned long long)j0 * p0.y;
#pragma unroll
          for (int r = 0; r < R; ++r)
            off[r] = bin_of_phase(f0 + (unsigned long long)r * p0.y, M) * T8 + (unsigned)r * MT8;
        }
        A2 aw = sAW[0];
        ulonglong2 pdn = sPD[cnt > 1 ? 1 : 0];
        A2 awn = sAW[cnt > 1 ? 1 : 0];
        for (int i = 0; i < cnt; ++i) {
          const int i2 = (i + 2 < cnt) ? i + 2 : cnt - 1;
          const ulonglong2 pdnn = sPD[i2];
          const A2 awnn = sAW[i2];
          A2 v[R];
#pragma unroll
          for (int r = 0; r < R; ++r) v[r] = *reinterpret_cast<const A2*>(my_bins + off[r]);
          const unsigned long long fn = pdn.x + (unsigned long long)j0 * pdn.y;
          unsigned offn[R];
#pragma unroll
          for (int r = 0; r < R; ++r)
            offn[r] = bin_of_phase(fn + (unsigned long long)r * pdn.y, M) * T8 + (unsigned)r * MT8;
#pragma unroll
          for (int r = 0; r < R; ++r) *reinterpret_cast<A2*>(my_bins + off[r]) = acc_add(v[r], aw);
#pragma unroll
          for (int r = 0; r < R; ++r) off[r] = offn[r];
          aw = awn;
          pdn = pdnn;
          awn = awnn;
        }
      } else {
        ulonglong2 pd = sPD[0];
        A2 aw = sAW[0];
#pragma unroll 2
        for (int i = 0; i < cnt; ++i) {
          const int in = (i + 1 < cnt) ? i + 1 : i;
          const ulonglong2 pdn = sPD[in];
          const A2 awn = sAW[in];
          // the R phases are independent multiply-adds (no serial chain of 64-bit adds)
          const unsigned long long phi0 = pd.x + (unsigned long long)j0 * pd.y;
          unsigned off[R];
#pragma unroll
          for (int r = 0; r < R; ++r)
            off[r] = bin_of_phase(phi0 + (unsigned long long)r * pd.y, M) * T8 + (unsigned)r * MT8;
          A2 v[R];
#pragma unroll
          for (int r = 0; r < R; ++r) v[r] = *reinterpret_cast<const A2*>(my_bins + off[r]);
#pragma unroll
          for (int r = 0; r < R; ++r) *reinterpret_cast<A2*>(my_bins + off[r]) = acc_add(v[r], aw);
          pd = pdn;
          aw = awn;
        }
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
          m = m < M ? m : M - 1u;
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
        k = k < 0 ? 0 : (k >= b.F ? b.F - 1 : k);
        fr[r] = args.freqs[k];
      }
      for (int i = 0; i < cnt; ++i) {
        const double ti = __longlong_as_double((long long)sPD[i].x);
        const A2 aw = sAW[i];
        unsigned off[R];
#pragma unroll
        for (int r = 0; r < R; ++r) off[r] = bin_of_phase(phase_fixed64(ti, fr[r]), M) * T8 + (unsigned)r * MT8;
        A2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = *reinterpret_cast<const A2*>(my_bins + off[r]);
#pragma unroll
        for (int r = 0; r < R; ++r) *reinterpret_cast<A2*>(my_bins + off[r]) = acc_add(v[r], aw);
      }
    }
    __syncthreads();
  }
}

// Step 4: the local maxima among this tile's owned frequencies (or every owned
// frequency in raw mode), ranked into the running top list topS/topI. The
// ranking key of frequency k is (k << key_shift) | extra[r].
template <int R, typename A>
__device__ __forceinline__ void tile_peaks(const TileArgs& args, const Block<A>& b, const A (&S)[R],
                                           const int (&extra)[R], int key_shift, int64_t s, const WorkItem& wi,
                                           double* topS, int* topI) {
  const int lane = b.lane, warp = b.warp, kk = b.kk, W = b.W;
  A left = __shfl_up_sync(0xffffffffu, S[R - 1], 1);
  A right = __shfl_down_sync(0xffffffffu, S[0], 1);
  A* const aedges = reinterpret_cast<A*>(b.edges);
  if (lane == 0) aedges[2 * warp] = S[0];
  if (lane == 31) aedges[2 * warp + 1] = S[R - 1];
  __syncthreads();
  if (lane == 0) left = (warp > 0) ? aedges[2 * warp - 1] : (A)-INFINITY;
  if (lane == 31) right = (warp + 1 < b.nwarps) ? aedges[2 * warp + 2] : (A)-INFINITY;
  const A thr = (topI[kk - 1] >= 0) ? (A)topS[kk - 1] : (A)-INFINITY;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int j = (int)b.j0 + r;
    const int64_t k = s + j;
    const bool owned = j > 0 && j < W - 1 && k >= wi.f_lo && k < wi.f_hi;
    const A prev = (r > 0) ? S[r > 0 ? r - 1 : 0] : left;
    const A next = (r < R - 1) ? S[r < R - 1 ? r + 1 : 0] : right;
    const bool peak = args.peak_raw ? owned : (owned && S[r] > prev && S[r] >= next);
    if (peak && S[r] > thr) {
      const int slot = atomicAdd(&b.misc[1], 1);
      b.candS[slot] = (double)S[r];
      b.candI[slot] = (int)((k << key_shift) | extra[r]);
    }
  }
  __syncthreads();
  const int cnt = b.misc[1];
  if (cnt > 0) {
    if (warp == 0) warp_merge_topk(topS, topI, kk, b.candS, b.candI, cnt, lane);
    __syncthreads();
    if (b.tid == 0) b.misc[1] = 0;
  }
  __syncthreads();
}

// Item prologue shared by both kernels: invalid curves produce NaN / empty
// candidates (returns false); otherwise the largest |t| of the curve (sets the
// grid-linearity tolerance) and cleared top lists.
template <typename A>
__device__ __forceinline__ bool item_begin(const TileArgs& args, const Block<A>& b, const WorkItem& wi, int64_t base,
                                           int64_t n, bool grid_bad, int groups, double& tm) {
  const int T = b.T, tid = b.tid, kk = b.kk;
  const int64_t F = b.F, c = wi.curve;
  if (grid_bad || args.curve_bad[c]) {
    if (args.S_out)
      for (int g = 0; g < groups; ++g)
        for (int64_t q = wi.f_lo + tid; q < wi.f_hi; q += T)
          args.S_out[(c * groups + g) * F + q] = __longlong_as_double(0x7ff8000000000000ll);
    if (kk > 0)
      for (int g = 0; g < groups; ++g)
        for (int q = tid; q < kk; q += T) {
          args.cand_S[(g * args.group_rows + wi.slot) * kk + q] = -INFINITY;
          args.cand_idx[(g * args.group_rows + wi.slot) * kk + q] = -1;
        }
    __syncthreads();
    return false;
  }
  double m = 0.0;
  for (int64_t i = tid; i < n; i += T) m = fmax(m, fabs(args.t[base + i]));
  m = warp_max(m);
  if (b.lane == 0) b.red[b.warp] = m;
  for (int q = tid; q < kk * groups; q += T) {
    const int g = q / kk, j = q % kk;
    b.topS[g * FPW_MAX_TOPK + j] = -INFINITY;
    b.topI[g * FPW_MAX_TOPK + j] = -1;
  }
  if (tid == 0) b.misc[1] = 0;
  __syncthreads();
  tm = 0.0;
  for (int w = 0; w < b.nwarps; ++w) tm = fmax(tm, b.red[w]);
  return true;
}

template <typename A>
__device__ __forceinline__ void item_end(const TileArgs& args, const Block<A>& b, const WorkItem& wi, int groups) {
  const int kk = b.kk;
  if (kk > 0)
    for (int q = b.tid; q < kk * groups; q += b.T) {
      const int g = q / kk, j = q % kk;
      args.cand_S[(g * args.group_rows + wi.slot) * kk + j] = b.topS[g * FPW_MAX_TOPK + j];
      args.cand_idx[(g * args.group_rows + wi.slot) * kk + j] = b.topI[g * FPW_MAX_TOPK + j];
    }
  __syncthreads();
}

template <int R, int PHASE, typename A>
__global__ void __launch_bounds__(512) tile_kernel(const TileArgs args) {
  using A2 = typename Acc2<A>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const Block<A> b = make_block<R, A>(smem, args);
  const int64_t F = b.F;
  const bool grid_bad = (*(volatile unsigned*)args.status & kStatusGrid) != 0u;
  const A cal = (A)args.inv_alpha2;

  // bins start at zero; every reduce leaves them zero again
  for (int q = 0; q < R * b.M; ++q) {
    A2 z;
    acc_zero(z);
    *reinterpret_cast<A2*>(b.my_bins + (size_t)q * b.T8) = z;
  }

  for (;;) {
    if (b.tid == 0) b.misc[0] = (int)atomicAdd(args.counter, 1u);
    __syncthreads();
    const int it = b.misc[0];
    if (it >= args.nitems) break;
    const WorkItem wi = args.items[it];
    const int c = wi.curve;
    int64_t base = 0, n = args.n_single;
    if (args.offsets) {
      base = args.offsets[c];
      n = args.offsets[c + 1] - base;
    }
    double tm;
    if (!item_begin(args, b, wi, base, n, grid_bad, 1, tm)) continue;
    const bool resident = n <= b.NC;
    bool staged_lin = false;

    for (int64_t s = (int64_t)wi.f_lo - 1; s + 1 < wi.f_hi; s += b.W - 2) {
      const int64_t a = s < 0 ? 0 : s;
      const double fa = args.freqs[a];
      const bool lin = tile_is_linear<R>(args, b, s, a, fa, tm);
      accumulate_tile<R, PHASE, A>(args, b, s, a, fa, lin, resident && staged_lin && lin, staged_lin, base, n);

      // reduce to S (and clear the bins for the next tile); S and the peak test
      // stay in the accumulation type (no binary64 work for FP32 sums)
      A S[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        A acc = (A)0;
        unsigned char* col = b.my_bins + (size_t)r * b.MT8;
        for (int m = 0; m < b.M; ++m) {
          A2* p = reinterpret_cast<A2*>(col + (size_t)m * b.T8);
          const A2 v = *p;
          A2 z;
          acc_zero(z);
          *p = z;
          const A den = v.y + cal;
          acc += (den > (A)0) ? quotient(v.x * v.x, den) : (A)0;
        }
        const int64_t k = s + (int64_t)b.j0 + r;
        S[r] = (k >= 0 && k < F) ? acc : (A)-INFINITY;
      }
      // dense output of owned frequencies
      if (args.S_out) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int j = (int)b.j0 + r;
          const int64_t k = s + j;
          if (j > 0 && j < b.W - 1 && k >= wi.f_lo && k < wi.f_hi) args.S_out[(int64_t)c * F + k] = (double)S[r];
        }
      }
      if (b.kk > 0) {
        int zero[R];
#pragma unroll
        for (int r = 0; r < R; ++r) zero[r] = 0;
        tile_peaks<R, A>(args, b, S, zero, 0, s, wi, b.topS, b.topI);
      } else {
        __syncthreads();
      }
    }
    item_end(args, b, wi, 1);
  }
}

// Several M from one M_max pass (Section 3.4): the kernel accumulates M_max
// bins; for each requested group g (M = M_max / g) it reports, per frequency,
// the largest S over the g bin offsets and that offset (ranking key
// (k << 6) | offset). FP32 sums.
template <int R, int PHASE>
__global__ void __launch_bounds__(512) tile_kernel_multi(const TileArgs args) {
  using A = float;
  using A2 = float2;
  extern __shared__ __align__(16) unsigned char smem[];
  const Block<A> b = make_block<R, A>(smem, args);
  const int64_t F = b.F;
  const int Mx = b.M, ng = args.ngroups;
  const bool grid_bad = (*(volatile unsigned*)args.status & kStatusGrid) != 0u;
  const A cal = (A)args.inv_alpha2;

  for (int q = 0; q < R * Mx; ++q) *reinterpret_cast<A2*>(b.my_bins + (size_t)q * b.T8) = make_float2(0.f, 0.f);

  for (;;) {
    if (b.tid == 0) b.misc[0] = (int)atomicAdd(args.counter, 1u);
    __syncthreads();
    const int it = b.misc[0];
    if (it >= args.nitems) break;
    const WorkItem wi = args.items[it];
    const int c = wi.curve;
    int64_t base = 0, n = args.n_single;
    if (args.offsets) {
      base = args.offsets[c];
      n = args.offsets[c + 1] - base;
    }
    double tm;
    if (!item_begin(args, b, wi, base, n, grid_bad, ng, tm)) continue;
    const bool resident = n <= b.NC;
    bool staged_lin = false;

    for (int64_t s = (int64_t)wi.f_lo - 1; s + 1 < wi.f_hi; s += b.W - 2) {
      const int64_t a = s < 0 ? 0 : s;
      const double fa = args.freqs[a];
      const bool lin = tile_is_linear<R>(args, b, s, a, fa, tm);
      accumulate_tile<R, PHASE, A>(args, b, s, a, fa, lin, resident && staged_lin && lin, staged_lin, base, n);

      // inclusive prefix sums Q[m] of the M_max bins, in place, per r
      float2 total[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        A2* col = reinterpret_cast<A2*>(b.my_bins + (size_t)r * b.MT8);
        const int st = b.T;  // stride between bins, in A2 units
        A2 run = make_float2(0.f, 0.f);
        for (int m = 0; m < Mx; ++m) {
          run = acc_add(run, col[m * st]);
          col[m * st] = run;
        }
        total[r] = run;
      }
      for (int g = 0; g < ng; ++g) {
        const int gs = args.group_g[g], Mg = Mx / gs;
        A S[R];
        int off[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const A2* col = reinterpret_cast<const A2*>(b.my_bins + (size_t)r * b.MT8);
          const int st = b.T;
          A best = (A)-INFINITY;
          int bo = 0;
          for (int o = 0; o < gs; ++o) {
            A acc = (A)0;
            for (int j = 0; j < Mg; ++j) {
              const int p0 = j * gs + o, p1 = p0 + gs - 1;
              A2 w;
              if (p1 < Mx) {
                w = col[p1 * st];
                if (p0 > 0) w = acc_sub(w, col[(p0 - 1) * st]);
              } else {  // the window wraps past bin M_max - 1 (then p0 >= 1)
                w = acc_add(acc_sub(total[r], col[(p0 - 1) * st]), col[(p1 - Mx) * st]);
              }
              const A den = w.y + cal;
              acc += (den > (A)0) ? quotient(w.x * w.x, den) : (A)0;
            }
            if (acc > best) {
              best = acc;
              bo = o;
            }
          }
          const int64_t k = s + (int64_t)b.j0 + r;
          S[r] = (k >= 0 && k < F) ? best : (A)-INFINITY;
          off[r] = bo;
        }
        if (args.S_out) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int j = (int)b.j0 + r;
            const int64_t k = s + j;
            if (j > 0 && j < b.W - 1 && k >= wi.f_lo && k < wi.f_hi)
              args.S_out[((int64_t)c * ng + g) * F + k] = (double)S[r];
          }
        }
        if (b.kk > 0) tile_peaks<R, A>(args, b, S, off, 6, s, wi, b.topS + g * FPW_MAX_TOPK, b.topI + g * FPW_MAX_TOPK);
      }
      // clear the bins for the next tile
#pragma unroll
      for (int r = 0; r < R; ++r) {
        A2* col = reinterpret_cast<A2*>(b.my_bins + (size_t)r * b.MT8);
        for (int m = 0; m < Mx; ++m) col[m * b.T] = make_float2(0.f, 0.f);
      }
      __syncthreads();
    }
    item_end(args, b, wi, ng);
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

template <int R, int PHASE>
const void* multi_fn() {
  return reinterpret_cast<const void*>(&tile_kernel_multi<R, PHASE>);
}

const void* pick(int R, int phase_mode, bool acc64, bool multi) {
  const bool fp32p = phase_mode == FPW_PHASE_FP32;
#define FPW_PICK(RR)                                                                                           \
  if (R == RR) {                                                                                               \
    if (multi) return fp32p ? multi_fn<RR, FPW_PHASE_FP32>() : multi_fn<RR, FPW_PHASE_FIXED64>();              \
    if (acc64) return fp32p ? tile_fn<RR, FPW_PHASE_FP32, double>() : tile_fn<RR, FPW_PHASE_FIXED64, double>(); \
    return fp32p ? tile_fn<RR, FPW_PHASE_FP32, float>() : tile_fn<RR, FPW_PHASE_FIXED64, float>();             \
  }
  FPW_PICK(1)
  FPW_PICK(2)
  FPW_PICK(4)
  FPW_PICK(8)
#undef FPW_PICK
  return nullptr;
}

}  // namespace

size_t tile_smem_bytes(int T, int R, int M, int NC, int /*k*/, bool accum64, int ngroups) {
  return tile_layout(T, R, M, NC, accum64, ngroups).total;
}

bool tile_supported_R(int R) { return R == 1 || R == 2 || R == 4 || R == 8; }

cudaError_t tile_init_attributes(int max_smem) {
  for (int R : {1, 2, 4, 8})
    for (int ph : {FPW_PHASE_FIXED64, FPW_PHASE_FP32})
      for (int v : {0, 1, 2}) {
        cudaError_t e = cudaFuncSetAttribute(pick(R, ph, v == 1, v == 2), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             max_smem);
        if (e != cudaSuccess) return e;
      }
  return cudaSuccess;
}

int tile_max_blocks_per_sm(int R, int phase_mode, bool accum64, int T, size_t smem, bool multi) {
  const void* fn = pick(R, phase_mode, accum64, multi);
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
  const void* fn = pick(s.R, phase_mode, accum64, a.ngroups > 0);
  if (!fn) return cudaErrorInvalidValue;
  void* params[] = {const_cast<TileArgs*>(&a)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(s.threads), params, s.smem, st);
}

}  // namespace fpw
