// Device templates of the persistent FPW tile kernels: Eq. 1 (Section 2) for
// every (curve, frequency) of a work list, with the per-curve top-k peaks of
// Section 3.5; and the same with several bin counts M = M_max / g derived from
// one M_max pass (Section 3.4). The kernels are instantiated in several
// translation units (fpw_tile_*.cu) so that they compile in parallel; the host
// side (shapes, launches) is fpw_tile.cu.
//
// Work decomposition
//   A work item is (curve c, frequency segment [f_lo, f_hi)). Thread blocks pop
//   items from a global counter (items are sorted by cost, longest first).
//   Within an item the segment is swept in tiles of W = T * R consecutive
//   frequencies: thread j owns tile positions j*R + r (r < R). Tiles overlap by
//   two frequencies so that every owned frequency has both neighbours in the
//   same tile (needed for the local-maximum test of the peak finder); tile
//   starts sit at q*(W-2) - 1 for integer q, whatever the item's segment.
//
// Per tile
//   1. Anchor: for each observation, Phi_s = frac(t_i * f_s) as a 64-bit
//      fixed-point fraction from the exact integer product of the binary64
//      significands, and the step D_i = frac(t_i * df) (df = grid spacing).
//      Both are staged in shared memory with the prep kernel's weights
//      (a_i = x_i w_i, w_i).
//   2. Hot loop (per observation, per thread, per r): Phi = Phi_s + (j*R + r) D_i
//      (mod 2^64), bin m = floor(M * Phi_hi / 2^32), A_m += a_i, B_m += w_i in a
//      thread-private [r][m][thread] bin array in shared memory (bank = lane,
//      so conflict-free), all R loads issued before the R stores; every thread
//      reads each staged observation (a warp-uniform broadcast).
//   3. Reduce: S = sum_m A_m^2 / (B_m + 1/alpha^2), empty bins contribute 0.
//      Several-M kernel: in-place prefix sums of the M_max bins, then for each
//      group g the windows of g consecutive bins (circularly) for every offset;
//      S_g(f) is the largest S over the g offsets, and that offset is kept.
//   4. Peaks: local maxima among owned frequencies, merged into the item's
//      running top-k (shared memory), written as candidates at the item's end.
//
// Grids that are not linear to within kGridTolCycles over a tile fall back to a
// direct exact anchor per (observation, frequency).
//
// Bin sums (policy P): FP32 pairs (A, B); binary64 pairs; or FP32 pairs with
// compensation terms (A, B, cA, cB), where each addition is an exact two-sum
// whose rounding error, plus the low part of the staged term, goes to the
// compensation term (the weights are staged as hi + lo FP32 pairs), so the
// sums carry about 48 significant bits; each bin's term is then taken from
// hi + lo rounded once to FP32, and S is accumulated in binary64.
//
// DUMP instantiations additionally write the bin m of every (observation,
// owned frequency k) with bins_k0 <= k < bins_k1 to args.bins_out, from the
// same arithmetic as the sums (bin-identity checks of the product kernel).
#pragma once
#include <math.h>

#include "fpw_internal.cuh"

namespace fpw {

// Per-translation-unit kernel getters (fpw_tile_*.cu).
const void* tile_fn_f32(int R, int phase_mode, bool dump);
const void* tile_fn_f32_odd(int R, int phase_mode, bool dump);  // R = 3, 5, 6
const void* tile_fn_f64(int R, int phase_mode, bool dump);
const void* tile_fn_comp(int R, int phase_mode, bool dump);
const void* tile_fn_multi(int R, int phase_mode, int spec);  // spec: multi_spec_of(), 0 = generic

struct TileLayout {
  size_t bins, pd, aw, candS, candI, topS, topI, edges, red, misc, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared-memory carve-up of one block: bins [R][M][T] of bin_bytes, the staged
// {Phi, D} (16 B) and weights (bin_bytes) of NC observations plus two padding
// records (read by the hot loop's prefetch past a chunk's last observation,
// never used), peak scratch.
__host__ __device__ inline TileLayout tile_layout(int T, int R, int M, int NC, size_t bin_bytes, int ngroups) {
  const size_t W = (size_t)T * R;
  const size_t tops = (size_t)(ngroups > 1 ? ngroups : 1) * FPW_MAX_TOPK;
  TileLayout L;
  size_t o = 0;
  L.bins = o;
  o = align16(o + (size_t)R * M * T * bin_bytes);
  L.pd = o;
  o = align16(o + (size_t)(NC + 2) * 16);
  L.aw = o;
  o = align16(o + (size_t)(NC + 2) * bin_bytes);
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

#ifdef __CUDACC__
namespace {

// ---- accumulation policies ----------------------------------------------
struct AccF32 {  // FP32 (A, B)
  using Bin = float2;
  using In = float2;  // (a, w)
  using S = float;
};
struct AccF64 {  // binary64 (A, B)
  using Bin = double2;
  using In = double2;
  using S = double;
};
struct AccComp {  // FP32 (A, B) with compensation (cA, cB): float4 {A, B, cA, cB}
  using Bin = float4;
  using In = float4;  // {a_hi, w_hi, a_lo, w_lo}
  using S = double;
};

__device__ __forceinline__ unsigned long long pack2(float2 a) {
  unsigned long long x;
  asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
  return x;
}
__device__ __forceinline__ float2 unpack2(unsigned long long z) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(z));
  return r;
}

__device__ __forceinline__ float2 bin_add(float2 v, float2 x) { return f2add(v, x); }
__device__ __forceinline__ double2 bin_add(double2 v, double2 x) { return make_double2(v.x + x.x, v.y + x.y); }
// Compensated: (s, e) = TwoSum(v.AB, x.hi) exactly (s + e = v.AB + x.hi), then
// c += e + x.lo. Packed FP32 pairs handle A and B together.
__device__ __forceinline__ float4 bin_add(float4 v, float4 x) {
  const unsigned long long a = pack2(make_float2(v.x, v.y)), b = pack2(make_float2(x.x, x.y));
  const unsigned long long c = pack2(make_float2(v.z, v.w)), lo = pack2(make_float2(x.z, x.w));
  unsigned long long s, bb, t1, t2, t3, e, c1, c2;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s) : "l"(a), "l"(b));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(bb) : "l"(s), "l"(a));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t1) : "l"(s), "l"(bb));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t2) : "l"(a), "l"(t1));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t3) : "l"(b), "l"(bb));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(e) : "l"(t2), "l"(t3));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(c1) : "l"(e), "l"(lo));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(c2) : "l"(c), "l"(c1));
  const float2 sv = unpack2(s), cv = unpack2(c2);
  return make_float4(sv.x, sv.y, cv.x, cv.y);
}

__device__ __forceinline__ void bin_zero(float2& v) { v = make_float2(0.f, 0.f); }
__device__ __forceinline__ void bin_zero(double2& v) { v = make_double2(0.0, 0.0); }
__device__ __forceinline__ void bin_zero(float4& v) { v = make_float4(0.f, 0.f, 0.f, 0.f); }

// One bin's term A^2 / (B + 1/alpha^2) of Eq. 1; a bin whose denominator is 0 contributes 0.
// FP32: the reciprocal-based quotient (2 ulp), branch-free (a branch to a
// correctly rounded division for out-of-range denominators kept the compiler
// from overlapping the terms of the reduce); a denominator outside
// [2^-100, 2^100] is scaled by 2^-+64 into that range first, the numerator
// alike, so the reciprocal stays accurate. Binary64: correctly rounded.
__device__ __forceinline__ float bin_term(float2 v, float cal) {
  const float den = v.y + cal;
  const float sc = den > 0x1p+100f ? 0x1p-64f : (den < 0x1p-100f ? 0x1p+64f : 1.0f);
  const float q = __fdividef((v.x * v.x) * sc, den * sc);
  return (den > 0.f) ? q : 0.f;
}
__device__ __forceinline__ double bin_term(double2 v, double cal) {
  const double den = v.y + cal;
  return (den > 0.0) ? v.x * v.x / den : 0.0;
}
// Compensated: the sums' value hi + lo rounded once to FP32 (the compensation
// already holds their rounding error), the term as in the FP32 policy (about
// 3e-7 relative), S accumulated in binary64. A binary64 division per bin took
// 28 % of the kernel's time at M = 20 and 44 % at M = 50.
__device__ __forceinline__ double bin_term(float4 v, double cal) {
  return (double)bin_term(make_float2(v.x + v.z, v.y + v.w), (float)cal);
}

__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Order-preserving map of a double to an unsigned integer (larger value, larger
// image), and its inverse.
__device__ __forceinline__ unsigned long long rank_bits(double s) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(s);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_rank_bits(unsigned long long r) {
  return __longlong_as_double((long long)((r >> 63) ? (r & 0x7fffffffffffffffull) : ~r));
}

// Selects the best kk entries of (top list) + (candidate list) into the top
// list, ranked by S descending then key ascending. Executed by one warp.
// Entries with key < 0 are empty. kk <= FPW_MAX_TOPK (two results per lane).
// Round q takes the best entry ranked after round q-1's pick (keys are unique
// within an item, so no entry needs marking): each lane's best over its
// strided share, then the warp's from three redux.sync maxima over (S's
// order-preserving high word, its low word, the inverted key).
__device__ void warp_merge_topk(double* topS, int* topI, int kk, double* cS, int* cI, int cnt, int lane) {
  double keepS[2] = {-INFINITY, -INFINITY};
  int keepI[2] = {-1, -1};
  const int pool = kk + cnt;
  unsigned long long prev_r = 0ull;
  unsigned prev_k = 0u;
  for (int q = 0; q < kk; ++q) {
    unsigned long long br = 0ull;  // 0: nothing (no double maps to 0 here)
    unsigned bk = 0u;
    for (int e = lane; e < pool; e += 32) {
      const int i = (e < kk) ? topI[e] : cI[e - kk];
      if (i < 0) continue;
      const unsigned long long r = rank_bits((e < kk) ? topS[e] : cS[e - kk]);
      const unsigned kx = ~(unsigned)i;
      const bool after = (q == 0) || r < prev_r || (r == prev_r && kx < prev_k);
      if (after && (r > br || (r == br && kx > bk))) {
        br = r;
        bk = kx;
      }
    }
    const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(br >> 32));
    const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(br >> 32) == hi ? (unsigned)br : 0u);
    const unsigned long long wr = ((unsigned long long)hi << 32) | lo;
    const unsigned wk = __reduce_max_sync(0xffffffffu, br == wr ? bk : 0u);
    if (wr == 0ull) break;  // every entry taken
    prev_r = wr;
    prev_k = wk;
    if (lane == (q & 31)) {
      keepS[q >> 5] = from_rank_bits(wr);
      keepI[q >> 5] = (int)~wk;
    }
  }
  __syncwarp();
  for (int q = lane; q < kk; q += 32) {
    topS[q] = keepS[q >> 5];
    topI[q] = keepI[q >> 5];
  }
  __syncwarp();
}

// Per-block view of shared memory and the constants every stage needs.
template <class P>
struct Block {
  using Bin = typename P::Bin;
  using In = typename P::In;
  unsigned char* my_bins;    // this thread's column of the [r][m][thread] bin array
  ulonglong2* sPD;           // staged {Phi_s, D} per observation
  In* sAW;                   // staged weights per observation
  double* candS;
  int* candI;
  double* topS;              // [groups][FPW_MAX_TOPK]
  int* topI;
  double* edges;
  double* red;
  int* misc;
  int T, tid, lane, warp, nwarps, M, NC, kk, W;
  unsigned T8, MT8, j0;      // T8: bytes between bins of a column; MT8: between its R frequencies
  int64_t F;
  double df;
};

template <int R, class P>
__device__ __forceinline__ Block<P> make_block(unsigned char* smem, const TileArgs& args) {
  using Bin = typename P::Bin;
  Block<P> b;
  b.T = blockDim.x;
  b.tid = threadIdx.x;
  b.lane = b.tid & 31;
  b.warp = b.tid >> 5;
  b.nwarps = b.T >> 5;
  b.M = args.M;
  b.NC = args.obs_chunk;
  b.kk = args.k;
  b.W = b.T * R;
  const TileLayout L = tile_layout(b.T, R, b.M, b.NC, sizeof(Bin), args.ngroups);
  b.my_bins = smem + L.bins + (size_t)b.tid * sizeof(Bin);
  b.sPD = reinterpret_cast<ulonglong2*>(smem + L.pd);
  b.sAW = reinterpret_cast<typename P::In*>(smem + L.aw);
  b.candS = reinterpret_cast<double*>(smem + L.candS);
  b.candI = reinterpret_cast<int*>(smem + L.candI);
  b.topS = reinterpret_cast<double*>(smem + L.topS);
  b.topI = reinterpret_cast<int*>(smem + L.topI);
  b.edges = reinterpret_cast<double*>(smem + L.edges);
  b.red = reinterpret_cast<double*>(smem + L.red);
  b.misc = reinterpret_cast<int*>(smem + L.misc);
  b.T8 = (unsigned)b.T * (unsigned)sizeof(Bin);
  b.MT8 = (unsigned)b.M * b.T8;
  b.j0 = (unsigned)b.tid * R;
  b.F = args.nfreq;
  b.df = (b.F > 1) ? (args.freqs[b.F - 1] - args.freqs[0]) / (double)(b.F - 1) : 0.0;
  return b;
}

// The two padding records after the staged chunk hold zeros (defined values
// for the prefetch that reads them; made visible by the first item's barrier).
template <class P>
__device__ __forceinline__ void zero_padding(const Block<P>& b) {
  if (b.tid < 2) {
    b.sPD[b.NC + b.tid] = make_ulonglong2(0ull, 0ull);
    typename P::In z;
    bin_zero(z);
    b.sAW[b.NC + b.tid] = z;
  }
}

// Is the grid linear over the tile starting at s? The precomputed per-tile
// deviation when available (tile starts sit at multiples of W-2, minus one),
// else checked here (block-wide).
template <int R, class P>
__device__ __forceinline__ bool tile_is_linear(const TileArgs& args, const Block<P>& b, int64_t s, int64_t a,
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

// DUMP: bins m[r] of observation `obs` (global index) at tile positions j + r.
template <int R>
__device__ __forceinline__ void dump_bins(const TileArgs& args, int W, int64_t s, const WorkItem& wi, int64_t obs,
                                          unsigned j, const unsigned (&m)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const unsigned jr = j + (unsigned)r;
    const int64_t k = s + (int64_t)jr;
    if (jr >= 1u && jr + 1u < (unsigned)W && k >= wi.f_lo && k < wi.f_hi && k >= args.bins_k0 && k < args.bins_k1)
      args.bins_out[(k - args.bins_k0) * args.bins_nobs + obs] = (int32_t)m[r];
  }
}

// Stages every observation chunk of the curve for the tile starting at s and
// accumulates its bins (steps 1 and 2). A curve that fits in one chunk keeps
// D_i and its weights staged across the tiles of an item (keep); only the
// anchor phase is then recomputed.
template <int R, int PHASE, class P, bool DUMP>
__device__ __forceinline__ void accumulate_tile(const TileArgs& args, const Block<P>& b, int64_t s, int64_t a,
                                                double fa, bool lin, bool keep, bool& staged_lin, int64_t base,
                                                int64_t n, const WorkItem& wi) {
  using Bin = typename P::Bin;
  using In = typename P::In;
  const int T = b.T, tid = b.tid, NC = b.NC;
  const unsigned M = (unsigned)b.M, T8 = b.T8, MT8 = b.MT8, j0 = b.j0;
  unsigned char* const my_bins = b.my_bins;
  ulonglong2* const sPD = b.sPD;
  In* const sAW = b.sAW;
  for (int64_t o = 0; o < n; o += NC) {
    const int cnt = (int)((n - o) < NC ? (n - o) : NC);
    for (int i = tid; i < cnt; i += T) {
      const double ti = args.t[base + o + i];
      if (keep) {
        const unsigned long long D = sPD[i].y;
        unsigned long long Pa = phase_fixed64(ti, fa);
        if (s < a) Pa -= D;  // tile starts one step before frequency 0
        sPD[i].x = Pa;
      } else {
        ulonglong2 pd;
        if (lin) {
          const unsigned long long D = phase_fixed64(ti, b.df);
          unsigned long long Pa = phase_fixed64(ti, fa);
          if (s < a) Pa -= D;
          pd = make_ulonglong2(Pa, D);
        } else {
          pd = make_ulonglong2((unsigned long long)__double_as_longlong(ti), 0ull);
        }
        sPD[i] = pd;
        sAW[i] = reinterpret_cast<const In*>(args.aw)[base + o + i];
      }
    }
    staged_lin = lin;
    __syncthreads();
    if (lin && PHASE == FPW_PHASE_FIXED64) {
      // Every thread reads each staged observation (a warp-uniform broadcast)
      // and adds it into its own column. The next observation's staged data
      // is loaded before this one's bin stores (the compiler cannot move it
      // there itself: both are shared memory), so the broadcast-load latency
      // overlaps the bin updates.
      if (R <= 2) {
        // Software-pipelined (measured faster at R <= 2, where the phase ->
        // bin -> offset chain is a larger share of each iteration; slower at
        // R = 4): the bins of observation i + 1 are computed while observation
        // i's bin loads are in flight, from staged data loaded one iteration
        // earlier. Same adds in the same order as the loop below.
        unsigned m[R];
        {
          const ulonglong2 p0 = sPD[0];
          const unsigned long long f0 = p0.x + (unsigned long long)j0 * p0.y;
#pragma unroll
          for (int r = 0; r < R; ++r) m[r] = bin_of_phase(f0 + (unsigned long long)r * p0.y, M);
        }
        In xv = sAW[0];
        ulonglong2 pdn = sPD[1];  // a padding record when cnt == 1
        In xn = sAW[1];
        for (int i = 0; i < cnt; ++i) {
          const ulonglong2 pdnn = sPD[i + 2];  // index <= cnt + 1 <= NC + 1: staged or padding
          const In xnn = sAW[i + 2];
          Bin v[R];
#pragma unroll
          for (int r = 0; r < R; ++r) v[r] = *reinterpret_cast<const Bin*>(my_bins + m[r] * T8 + (unsigned)r * MT8);
          const unsigned long long fn = pdn.x + (unsigned long long)j0 * pdn.y;
          unsigned mn[R];
#pragma unroll
          for (int r = 0; r < R; ++r) mn[r] = bin_of_phase(fn + (unsigned long long)r * pdn.y, M);
#pragma unroll
          for (int r = 0; r < R; ++r)
            *reinterpret_cast<Bin*>(my_bins + m[r] * T8 + (unsigned)r * MT8) = bin_add(v[r], xv);
          if (DUMP) dump_bins<R>(args, b.W, s, wi, base + o + i, j0, m);
#pragma unroll
          for (int r = 0; r < R; ++r) m[r] = mn[r];
          xv = xn;
          pdn = pdnn;
          xn = xnn;
        }
      } else {
        ulonglong2 pd = sPD[0];
        In xv = sAW[0];
#pragma unroll 2
        for (int i = 0; i < cnt; ++i) {
          const ulonglong2 pdn = sPD[i + 1];  // index <= cnt <= NC: staged or padding
          const In xn = sAW[i + 1];
          // the R phases are independent multiply-adds (no serial chain of 64-bit adds)
          const unsigned long long phi0 = pd.x + (unsigned long long)j0 * pd.y;
          unsigned m[R];
#pragma unroll
          for (int r = 0; r < R; ++r) m[r] = bin_of_phase(phi0 + (unsigned long long)r * pd.y, M);
          Bin v[R];
#pragma unroll
          for (int r = 0; r < R; ++r) v[r] = *reinterpret_cast<const Bin*>(my_bins + m[r] * T8 + (unsigned)r * MT8);
#pragma unroll
          for (int r = 0; r < R; ++r)
            *reinterpret_cast<Bin*>(my_bins + m[r] * T8 + (unsigned)r * MT8) = bin_add(v[r], xv);
          if (DUMP) dump_bins<R>(args, b.W, s, wi, base + o + i, j0, m);
          pd = pdn;
          xv = xn;
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
        const In xv = sAW[i];
        const float d32 = (float)(unsigned)(pd.y >> 32) * 0x1p-32f;
        unsigned m[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const unsigned long long pa = pd.x + (unsigned long long)da[r] * pd.y;
          const float p32 = (float)(unsigned)(pa >> 32) * 0x1p-32f;
          float p = fmaf(jr[r], d32, p32);
          p = p - floorf(p);
          unsigned mm = (unsigned)(p * (float)M);
          m[r] = mm < M ? mm : M - 1u;
        }
        Bin v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = *reinterpret_cast<const Bin*>(my_bins + m[r] * T8 + (unsigned)r * MT8);
#pragma unroll
        for (int r = 0; r < R; ++r)
          *reinterpret_cast<Bin*>(my_bins + m[r] * T8 + (unsigned)r * MT8) = bin_add(v[r], xv);
        if (DUMP) dump_bins<R>(args, b.W, s, wi, base + o + i, j0, m);
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
        const In xv = sAW[i];
        unsigned m[R];
#pragma unroll
        for (int r = 0; r < R; ++r) m[r] = bin_of_phase(phase_fixed64(ti, fr[r]), M);
        Bin v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = *reinterpret_cast<const Bin*>(my_bins + m[r] * T8 + (unsigned)r * MT8);
#pragma unroll
        for (int r = 0; r < R; ++r)
          *reinterpret_cast<Bin*>(my_bins + m[r] * T8 + (unsigned)r * MT8) = bin_add(v[r], xv);
        if (DUMP) dump_bins<R>(args, b.W, s, wi, base + o + i, j0, m);
      }
    }
    __syncthreads();
  }
}

// Step 4: the local maxima among this tile's owned frequencies (or every owned
// frequency in raw mode), ranked into the running top list topS/topI. The
// ranking key of frequency k is (k << key_shift) | extra[r].
template <int R, class P>
__device__ __forceinline__ void tile_peaks(const TileArgs& args, const Block<P>& b, const typename P::S (&S)[R],
                                           const int (&extra)[R], int key_shift, int64_t s, const WorkItem& wi,
                                           double* topS, int* topI) {
  using A = typename P::S;
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
template <class P>
__device__ __forceinline__ bool item_begin(const TileArgs& args, const Block<P>& b, const WorkItem& wi, int64_t base,
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

template <class P>
__device__ __forceinline__ void item_end(const TileArgs& args, const Block<P>& b, const WorkItem& wi, int groups) {
  const int kk = b.kk;
  if (kk > 0)
    for (int q = b.tid; q < kk * groups; q += b.T) {
      const int g = q / kk, j = q % kk;
      args.cand_S[(g * args.group_rows + wi.slot) * kk + j] = b.topS[g * FPW_MAX_TOPK + j];
      args.cand_idx[(g * args.group_rows + wi.slot) * kk + j] = b.topI[g * FPW_MAX_TOPK + j];
    }
  __syncthreads();
}

// (512, 1) sets the same 128-register ceiling as a bare 512-thread bound; with
// it the compiler gives every instantiation the registers it needs, where the
// bare bound led it to hold some to 64 registers and spill.
template <int R, int PHASE, class P, bool DUMP>
__global__ void __launch_bounds__(512, 1) tile_kernel(const TileArgs args) {
  using Bin = typename P::Bin;
  using A = typename P::S;
  extern __shared__ __align__(16) unsigned char smem[];
  const Block<P> b = make_block<R, P>(smem, args);
  const int64_t F = b.F;
  const bool grid_bad = (*(volatile unsigned*)args.status & kStatusGrid) != 0u;
  const A cal = (A)args.inv_alpha2;

  // bins start at zero; every reduce leaves them zero again
  for (int q = 0; q < R * b.M; ++q) {
    Bin z;
    bin_zero(z);
    *reinterpret_cast<Bin*>(b.my_bins + (size_t)q * b.T8) = z;
  }
  zero_padding(b);

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
      accumulate_tile<R, PHASE, P, DUMP>(args, b, s, a, fa, lin, resident && staged_lin && lin, staged_lin, base, n,
                                         wi);

      // reduce to S (and clear the bins for the next tile); S and the peak test
      // stay in the policy's reduce type
      A S[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        A acc = (A)0;
        unsigned char* col = b.my_bins + (size_t)r * b.MT8;
        Bin z;
        bin_zero(z);
        int m = 0;
        for (; m + 8 <= b.M; m += 8) {  // eight bins loaded before any is cleared: their loads overlap
          Bin v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = *reinterpret_cast<const Bin*>(col + (size_t)(m + u) * b.T8);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            *reinterpret_cast<Bin*>(col + (size_t)(m + u) * b.T8) = z;
            acc += bin_term(v[u], cal);
          }
        }
        for (; m < b.M; ++m) {
          Bin* p = reinterpret_cast<Bin*>(col + (size_t)m * b.T8);
          const Bin v = *p;
          *p = z;
          acc += bin_term(v, cal);
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
        tile_peaks<R, P>(args, b, S, zero, 0, s, wi, b.topS, b.topI);
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
// (k << 6) | offset). FP32 sums. At most 256 threads per block (the host
// rejects more): with that bound the compiler keeps the combination's
// registers (72-114) instead of spilling them, which it did at 40 registers
// under a 512-thread bound.
constexpr int kMultiMaxThreads = 256;
// Several-M combinations compiled for one M_max and three groups: the ones
// Section 3.4 suggests (M_max = 60 or 40, giving M = 20, 10 and 4) and the
// M = 20, 10, 5 split of M_max = 20. SPEC 0 is the generic combination.
template <int SPEC>
struct MultiSpec;
template <>
struct MultiSpec<1> {
  static constexpr int MX = 60, G0 = 3, G1 = 6, G2 = 15;
};
template <>
struct MultiSpec<2> {
  static constexpr int MX = 40, G0 = 2, G1 = 4, G2 = 10;
};
template <>
struct MultiSpec<3> {
  static constexpr int MX = 20, G0 = 1, G1 = 2, G2 = 4;
};

// One group's windows at bin m of the fixed combination: the window that ends
// at m, [m - g + 1, m], belongs to offset (m + 1) mod g; its sum is Q_m minus
// the prefix before its start (zero for the first window of offset 0).
template <int G, int M, int MX>
__device__ __forceinline__ void fixed_window(const float2 (&Q)[MX], float (&acc)[G], float cal) {
  if constexpr (M >= G) {
    acc[(M + 1) % G] += bin_term(f2sub(Q[M], Q[M - G]), cal);
  } else if constexpr (M == G - 1) {
    acc[0] += bin_term(f2sub(Q[M], make_float2(0.f, 0.f)), cal);
  }
}

// The wrapping window of each offset o >= 1, [M_max - g + o, M_max - 1] and
// [0, o - 1], added after the others; then the best offset (ties to the lower).
template <int G, int MX>
__device__ __forceinline__ void fixed_finish(const float2 (&Q)[MX], float (&acc)[G], float cal, float& best,
                                             int& bo) {
  const float2 total = Q[MX - 1];
#pragma unroll
  for (int o = 1; o < G; ++o) acc[o] += bin_term(bin_add(f2sub(total, Q[MX - G + o - 1]), Q[o - 1]), cal);
  best = -INFINITY;
  bo = 0;
#pragma unroll
  for (int o = 0; o < G; ++o)
    if (acc[o] > best) {
      best = acc[o];
      bo = o;
    }
}

template <int MX, int G0, int G1, int G2, int M>
__device__ __forceinline__ void fixed_step(float2 (&Q)[MX], float2 v, float2& run, float (&a0)[G0], float (&a1)[G1],
                                           float (&a2)[G2], float cal) {
  run = bin_add(run, v);
  Q[M] = run;
  fixed_window<G0, M, MX>(Q, a0, cal);
  fixed_window<G1, M, MX>(Q, a1, cal);
  fixed_window<G2, M, MX>(Q, a2, cal);
}

template <int MX, int G0, int G1, int G2, int C, int U>
__device__ __forceinline__ void fixed_chunk(float2 (&Q)[MX], const float2 (&v)[4], float2& run, float (&a0)[G0],
                                            float (&a1)[G1], float (&a2)[G2], float cal) {
  if constexpr (U < 4) {
    fixed_step<MX, G0, G1, G2, C * 4 + U>(Q, v[U], run, a0, a1, a2, cal);
    fixed_chunk<MX, G0, G1, G2, C, U + 1>(Q, v, run, a0, a1, a2, cal);
  }
}

// Chunk C of four bins: the next chunk's bins are loaded before this chunk's
// bins are cleared, so the loads of two chunks are in flight together.
template <int MX, int G0, int G1, int G2, int C>
__device__ __forceinline__ void fixed_chunks(float2* col, int st, float2 (&Q)[MX], float2 (&v)[4], float2& run,
                                             float (&a0)[G0], float (&a1)[G1], float (&a2)[G2], float cal) {
  if constexpr (C < MX / 4) {
    float2 vn[4];
    if constexpr (C + 1 < MX / 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) vn[u] = col[((C + 1) * 4 + u) * st];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) col[(C * 4 + u) * st] = make_float2(0.f, 0.f);
    fixed_chunk<MX, G0, G1, G2, C, 0>(Q, v, run, a0, a1, a2, cal);
    if constexpr (C + 1 < MX / 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = vn[u];
    }
    fixed_chunks<MX, G0, G1, G2, C + 1>(col, st, Q, v, run, a0, a1, a2, cal);
  }
}

// Several-M combination of one slot's M_max bins for a compiled (M_max, groups):
// one pass reads each bin once, clears it, forms the inclusive prefix sums Q_m
// in registers and adds every window that ends at bin m to its offset's sum;
// the windows that wrap past bin M_max - 1 are added last. The windows, terms
// and order of additions are those of the generic combination (in-place prefix
// sums, then per group and offset the windows in order, the wrapping one last),
// so S is the same bit for bit, while each bin costs one shared-memory read and
// one store instead of a read-modify-write for the prefix sums, a read per
// group and a clearing store.
template <int SPEC>
__device__ __forceinline__ void combine_fixed(float2* col, int st, float cal, float (&best)[3], int (&bo)[3]) {
  using SP = MultiSpec<SPEC>;
  constexpr int MX = SP::MX, G0 = SP::G0, G1 = SP::G1, G2 = SP::G2;
  static_assert(MX % 4 == 0 && MX % G0 == 0 && MX % G1 == 0 && MX % G2 == 0, "groups must divide M_max");
  float2 Q[MX];
  float a0[G0], a1[G1], a2[G2];
#pragma unroll
  for (int o = 0; o < G0; ++o) a0[o] = 0.f;
#pragma unroll
  for (int o = 0; o < G1; ++o) a1[o] = 0.f;
#pragma unroll
  for (int o = 0; o < G2; ++o) a2[o] = 0.f;
  float2 v[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) v[u] = col[u * st];
  float2 run = make_float2(0.f, 0.f);
  fixed_chunks<MX, G0, G1, G2, 0>(col, st, Q, v, run, a0, a1, a2, cal);
  fixed_finish<G0, MX>(Q, a0, cal, best[0], bo[0]);
  fixed_finish<G1, MX>(Q, a1, cal, best[1], bo[1]);
  fixed_finish<G2, MX>(Q, a2, cal, best[2], bo[2]);
}



template <int R, int PHASE, int SPEC>
__global__ void __launch_bounds__(kMultiMaxThreads, 2) tile_kernel_multi(const TileArgs args) {
  using P = AccF32;
  using A = float;
  using A2 = float2;
  extern __shared__ __align__(16) unsigned char smem[];
  const Block<P> b = make_block<R, P>(smem, args);
  const int64_t F = b.F;
  const int Mx = b.M, ng = args.ngroups;
  const bool grid_bad = (*(volatile unsigned*)args.status & kStatusGrid) != 0u;
  const A cal = (A)args.inv_alpha2;

  for (int q = 0; q < R * Mx; ++q) *reinterpret_cast<A2*>(b.my_bins + (size_t)q * b.T8) = make_float2(0.f, 0.f);
  zero_padding(b);

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
      accumulate_tile<R, PHASE, P, false>(args, b, s, a, fa, lin, resident && staged_lin && lin, staged_lin, base,
                                          n, wi);

      // the reported S of group g per owned frequency, and the peaks
      auto emit = [&](int g, const A (&S)[R], const int (&off)[R]) {
        if (args.S_out) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int j = (int)b.j0 + r;
            const int64_t k = s + j;
            if (j > 0 && j < b.W - 1 && k >= wi.f_lo && k < wi.f_hi)
              args.S_out[((int64_t)c * ng + g) * F + k] = (double)S[r];
          }
        }
        if (b.kk > 0) tile_peaks<R, P>(args, b, S, off, 6, s, wi, b.topS + g * FPW_MAX_TOPK, b.topI + g * FPW_MAX_TOPK);
      };
      if constexpr (SPEC != 0) {
        // compiled (M_max, groups): one pass per slot, bins cleared on the way
        A Sg[3][R];
        int offg[3][R];
#pragma unroll 1
        for (int r = 0; r < R; ++r) {  // one slot at a time: the pass holds its prefix sums in registers
          float best[3];
          int bo[3];
          combine_fixed<SPEC>(reinterpret_cast<A2*>(b.my_bins + (size_t)r * b.MT8), b.T, cal, best, bo);
          const int64_t k = s + (int64_t)b.j0 + r;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            Sg[q][r] = (k >= 0 && k < F) ? best[q] : (A)-INFINITY;
            offg[q][r] = bo[q];
          }
        }
#pragma unroll
        for (int g = 0; g < 3; ++g) emit(g, Sg[g], offg[g]);
      } else {
        // inclusive prefix sums Q[m] of the M_max bins, in place, per r; eight
        // bins are loaded before any of them is stored back, so the loads of a
        // chunk are in flight together (the bins of one thread form a dependent
        // chain otherwise: a load cannot pass the previous bin's store)
        float2 total[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          A2* col = reinterpret_cast<A2*>(b.my_bins + (size_t)r * b.MT8);
          const int st = b.T;  // stride between bins, in A2 units
          A2 run = make_float2(0.f, 0.f);
          int m = 0;
          for (; m + 8 <= Mx; m += 8) {
            A2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = col[(m + u) * st];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              run = bin_add(run, v[u]);
              col[(m + u) * st] = run;
            }
          }
          for (; m < Mx; ++m) {
            run = bin_add(run, col[m * st]);
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
              // window j spans bins [j gs + o, j gs + o + gs - 1]: its sum is
              // Q[end] - Q[start - 1], and its end is the next window's start - 1,
              // so one prefix value is read per window (carried in `prev`)
              const A2 q0 = (o > 0) ? col[(o - 1) * st] : make_float2(0.f, 0.f);
              A2 prev = q0;
              // the windows that end below bin M_max: independent loads (no
              // stores here), unrolled so that they issue together; the terms
              // are added in window order
              const int nin = (o > 0) ? Mg - 1 : Mg;
              const A2* e = col + (size_t)(o + gs - 1) * st;
#pragma unroll 4
              for (int j = 0; j < nin; ++j) {
                const A2 q = e[(size_t)j * gs * st];
                acc += bin_term(f2sub(q, prev), cal);
                prev = q;
              }
              // o >= 1: the last window wraps past bin M_max - 1 and ends at o - 1
              if (o > 0) acc += bin_term(bin_add(f2sub(total[r], prev), q0), cal);
              if (acc > best) {
                best = acc;
                bo = o;
              }
            }
            const int64_t k = s + (int64_t)b.j0 + r;
            S[r] = (k >= 0 && k < F) ? best : (A)-INFINITY;
            off[r] = bo;
          }
          emit(g, S, off);
        }
        // clear the bins for the next tile
#pragma unroll
        for (int r = 0; r < R; ++r) {
          A2* col = reinterpret_cast<A2*>(b.my_bins + (size_t)r * b.MT8);
          for (int m = 0; m < Mx; ++m) col[m * b.T] = make_float2(0.f, 0.f);
        }
      }
      __syncthreads();
    }
    item_end(args, b, wi, ng);
  }
}

}  // namespace
#endif  // __CUDACC__

}  // namespace fpw
