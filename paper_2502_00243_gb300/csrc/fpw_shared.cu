// Curves that share their observation times (Section 4 and the batch routine of
// Appendix D): the bins of every (observation, frequency) pair are the same for
// all curves, so per frequency the bin sums of a whole group of curves are one
// matrix product
//
//   D[(curve, part), (frequency, bin)] = sum_i  V[(curve, part), i] * H[i, (frequency, bin)]
//
// with V the per-observation values (part 0: a_i = x_i / sigma_i^2, part 1:
// w_i = 1 / sigma_i^2) and H the one-hot bin matrix (H[i, (f, m)] = 1 iff
// observation i falls in bin m at frequency f). That product runs on the
// tensor cores (tcgen05.mma kind::f16, FP32 accumulators in tensor memory):
//
// * V in fp16 with FP32-level precision: each value is scaled by a power of two
//   per curve and part (exact), then split v = hi + lo into two fp16 numbers;
//   hi and lo are adjacent entries of the K dimension, and the one-hot row of
//   the observation is duplicated for both, so the tensor core adds hi + lo
//   itself. Products with the one-hot entries are exact; sums are FP32.
// * H is built in shared memory for each chunk of 32 observations from exact
//   phases (phase_fixed64: the integer product of the binary64 significands),
//   so bins equal floor(M frac(t f)) except within 2^-32 of a cycle below an edge.
// * One CTA per SM (persistent over (group of 64 curves, frequency pass) work
//   items) holds two accumulators of 128 x N (N = frequencies per pass x M
//   <= 256) in 512 TMEM columns; V chunks arrive by bulk copy (TMA) into a
//   double buffer, H is double-buffered too, and the single issuing thread's
//   MMAs signal an mbarrier per buffer (tcgen05.commit).
// * The epilogue reads D with tcgen05.ld (lane = (curve, part) row), pairs the
//   two parts of a curve with one shuffle, and reduces S = sum_m A_m^2 / (B_m +
//   1/alpha^2) per frequency into a dense FP32 array; a per-curve top-k pass
//   follows.
//
// Every wait (mbarrier) is bounded by a clock limit; on expiry the kernel sets
// kStatusTimeout, waits (bounded) for its own copies and MMAs, frees its tensor
// memory and returns.
#include <cuda_fp16.h>
#include <math.h>

#include "fpw_shared.cuh"

namespace fpw {
namespace {

constexpr int kShCurves = 64;                   // curves per group
constexpr int kShRows = 128;                    // MMA M: (curve, part) rows
constexpr int kShObs = 32;                      // observations per chunk
constexpr int kShK = 2 * kShObs;                // K entries per chunk (hi, lo)
constexpr int kShKSteps = kShK / 16;            // MMA k-steps per chunk
constexpr int kShChunkBytes = kShRows * kShK * 2;  // V image of one chunk: 16 KB
constexpr int kShThreads = 256;
constexpr int kShNMax = 256;                    // MMA N limit (M = 128)
constexpr int kShHOperandMax = kShNMax * kShK * 2;   // one H operand of a chunk: 32 KB
constexpr int kShHSlotBytes = 2 * kShHOperandMax;    // two H operands (two accumulators)
constexpr int kShTmemCols = 512;
constexpr unsigned kOneOne = 0x3C003C00u;       // two fp16 1.0
constexpr long long kWaitClocks = 4000000000LL; // ~2 s at 2 GHz

// Shared-memory carve-up (bytes).
constexpr int kOffV = 0;                                   // 2 x 16 KB
constexpr int kOffH = kOffV + 2 * kShChunkBytes;           // 2 x 64 KB
constexpr int kOffBins = kOffH + 2 * kShHSlotBytes;        // bins of the chunk: [pass freq][32] bytes
constexpr int kMaxPassFreqs = 2 * kShNMax;                 // M = 1: 256 frequencies per accumulator
constexpr int kOffBar = kOffBins + kMaxPassFreqs * kShObs;
constexpr int kSmemBytes = kOffBar + 64;

// Byte offset of element (row r, k-entry q) of a K-major, unswizzled operand
// with R rows and kShK columns: one 16-column k-step after another; inside a
// k-step, 8-row x 16-byte core matrices, the two of a row group adjacent (the
// K-direction stride, 128 B) and row groups 256 B apart.
__host__ __device__ __forceinline__ uint32_t km_off(uint32_t r, uint32_t q, uint32_t R) {
  return (q >> 4) * (R * 32u) + (r >> 3) * 256u + ((q >> 3) & 1u) * 128u + (r & 7u) * 16u + (q & 7u) * 2u;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: unswizzled, K-direction core-matrix
// stride 128 B (leading byte offset), row-group stride 256 B (stride byte offset).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(256u >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version
  return d;
}

// Instruction descriptor, kind::f16: fp16 A and B (K-major), FP32 D, M x N.
__device__ __forceinline__ uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait for completion of phase `parity` of an mbarrier.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitClocks) return false;
  }
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------- prep
// One block per curve slot of the padded groups: validation, per-curve
// power-of-two scales, and the fp16 hi/lo image of (a, w) in the operand
// layout, one 16 KB chunk per (group, 32 observations).
__global__ void __launch_bounds__(256) shared_prep_kernel(const SharedArgs a) {
  __shared__ double red_a[8], red_w[8];
  __shared__ int red_bad[8];
  const int64_t c = blockIdx.x;  // padded curve slot
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = a.n;
  const bool real = c < a.ncurves;
  double amax = 0.0, wmax = 0.0;
  int bad = 0;
  if (real) {
    for (int64_t i = tid; i < n; i += blockDim.x) {
      const double s = a.sigma[c * n + i], x = a.x[c * n + i], t = a.t[i];
      const bool ok = isfinite(s) && isfinite(x) && isfinite(t) && s > 0.0;
      if (!ok) {
        bad = 1;
        continue;
      }
      const double w = 1.0 / (s * s);
      amax = fmax(amax, fabs(x * w));
      wmax = fmax(wmax, w);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (lane == 0) {
    red_a[warp] = amax;
    red_w[warp] = wmax;
    red_bad[warp] = bad;
  }
  __syncthreads();
  amax = 0.0;
  wmax = 0.0;
  bad = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
    amax = fmax(amax, red_a[q]);
    wmax = fmax(wmax, red_w[q]);
    bad |= red_bad[q];
  }
  // scale so that the largest magnitude lies in [2^14, 2^15): fp16 holds it
  // with room for the hi + lo split; an all-zero part keeps scale 1
  const int ea = amax > 0.0 ? 14 - ilogb(amax) : 0;
  const int ew = wmax > 0.0 ? 14 - ilogb(wmax) : 0;
  if (tid == 0) {
    a.inv_scale[2 * c] = real ? ldexpf(1.0f, -ea) : 0.0f;
    a.inv_scale[2 * c + 1] = real ? ldexpf(1.0f, -ew) : 0.0f;
    a.curve_bad[c] = (uint8_t)(real && bad);
    if (real && bad) atomicOr(a.status, kStatusData);
  }
  const int64_t g = c / kShCurves;
  const uint32_t row = (uint32_t)(c % kShCurves) * 2u;
  const bool zero = !real || bad;
  unsigned char* img = a.image + (size_t)g * (size_t)a.nchunks * kShChunkBytes;
  const int64_t npad = a.nchunks * kShObs;
  for (int64_t i = tid; i < npad; i += blockDim.x) {
    float av = 0.f, wv = 0.f;
    if (!zero && i < n) {
      const double s = a.sigma[c * n + i];
      const double w = 1.0 / (s * s);
      av = (float)ldexp(a.x[c * n + i] * w, ea);
      wv = (float)ldexp(w, ew);
    }
    const __half ah = __float2half_rn(av), wh = __float2half_rn(wv);
    const __half al = __float2half_rn(av - __half2float(ah)), wl = __float2half_rn(wv - __half2float(wh));
    unsigned char* ch = img + (size_t)(i / kShObs) * kShChunkBytes;
    const uint32_t q = 2u * (uint32_t)(i % kShObs);
    *reinterpret_cast<__half2*>(ch + km_off(row, q, kShRows)) = __halves2half2(ah, al);
    *reinterpret_cast<__half2*>(ch + km_off(row + 1u, q, kShRows)) = __halves2half2(wh, wl);
  }
  if (blockIdx.x == 0)
    for (int64_t q = tid; q < a.nfreq; q += blockDim.x)
      if (!isfinite(a.freqs[q])) atomicOr(a.status, kStatusGrid);
}

// ---------------------------------------------------------------- MMA kernel
__global__ void __launch_bounds__(kShThreads, 1) shared_mma_kernel(const SharedArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sV = smem + kOffV;
  unsigned char* sH = smem + kOffH;
  uint8_t* sBins = smem + kOffBins;
  uint64_t* bar_mma = reinterpret_cast<uint64_t*>(smem + kOffBar);  // [2]
  uint64_t* bar_v = bar_mma + 2;                                     // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar_mma + 4);
  int* s_abort = reinterpret_cast<int*>(tslot + 1);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int M = a.M, fpm = a.fpm, Nm = a.n_mma, FP = 2 * fpm, rows_used = fpm * M;
  const int64_t F = a.nfreq, n = a.n, nch = a.nchunks;
  const bool grid_bad = (*(volatile unsigned*)a.status & kStatusGrid) != 0u;
  const int64_t items = grid_bad ? 0 : a.ngroups * a.npass;
  const float cal = (float)a.inv_alpha2;

  if (tid == 0) {
    mbar_init(&bar_mma[0]);
    mbar_init(&bar_mma[1]);
    mbar_init(&bar_v[0]);
    mbar_init(&bar_v[1]);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(kShTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // H rows beyond fpm * M (padding up to the MMA's N) stay zero for good
  for (int e = tid; e < 2 * kShHSlotBytes / 16; e += kShThreads)
    reinterpret_cast<uint4*>(sH)[e] = make_uint4(0u, 0u, 0u, 0u);
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = mma_idesc(kShRows, Nm);

  // this thread's H rows (at most two: rows_used <= 2 x 256 over 256 threads... per operand)
  // row id e in [0, 2 * rows_used): operand e / rows_used, (j, m) within it
  int my_row_j[2], my_row_m[2];
  uint32_t my_row_off[2];
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int e = tid + kk * kShThreads;
    my_row_j[kk] = -1;
    my_row_m[kk] = 0;
    my_row_off[kk] = 0;
    if (e < 2 * rows_used) {
      const int op = e / rows_used, r = e % rows_used;
      my_row_j[kk] = op * fpm + r / M;  // pass-local frequency
      my_row_m[kk] = r % M;
      my_row_off[kk] = (uint32_t)(op * (Nm * kShK * 2)) + (uint32_t)(r >> 3) * 256u + (uint32_t)(r & 7) * 16u;
    }
  }

  uint32_t ph_mma[2] = {0u, 0u}, ph_v[2] = {0u, 0u};
  bool pend[2] = {false, false};
  bool abort = false;

  for (int64_t item = blockIdx.x; item < items && !abort; item += gridDim.x) {
    const int64_t g = item / a.npass, p = item % a.npass;
    const int64_t f0 = p * FP;
    const unsigned char* img = a.image + (size_t)g * (size_t)nch * kShChunkBytes;
    for (int64_t ch = 0; ch < nch; ++ch) {
      const int s = (int)(ch & 1);
      bool fail = false;
      if (pend[s]) {  // the MMAs of chunk ch - 2 read this buffer
        fail = !mbar_wait(&bar_mma[s], ph_mma[s]);
        ph_mma[s] ^= 1u;
        pend[s] = false;
      }
      if (__syncthreads_or(fail)) {
        abort = true;
        break;
      }
      if (tid == 0) bulk_load(sV + s * kShChunkBytes, img + (size_t)ch * kShChunkBytes, kShChunkBytes, &bar_v[s]);
      // bins of the chunk: pair (j, i) -> sBins[j * 32 + i]
      for (int e = tid; e < FP * kShObs; e += kShThreads) {
        const int j = e / kShObs, i = e % kShObs;
        const int64_t fi = f0 + j, oi = ch * kShObs + i;
        unsigned m = 0u;
        if (fi < F && oi < n) m = bin_of_phase(phase_fixed64(a.t[oi], a.freqs[fi]), (unsigned)M);
        sBins[e] = (uint8_t)m;
      }
      __syncthreads();
      // one-hot H: 16-byte pieces (4 observations x hi/lo) per (row, k-group)
      unsigned char* hs = sH + s * kShHSlotBytes;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        if (my_row_j[kk] < 0) continue;
        const uint32_t mrep = (uint32_t)my_row_m[kk] * 0x01010101u;
        const uint32_t* bw = reinterpret_cast<const uint32_t*>(sBins + my_row_j[kk] * kShObs);
#pragma unroll
        for (int q4 = 0; q4 < kShObs / 4; ++q4) {
          const uint32_t eq = __vcmpeq4(bw[q4], mrep);
          uint4 v;
          v.x = __byte_perm(eq, 0u, 0x0000u) & kOneOne;
          v.y = __byte_perm(eq, 0u, 0x1111u) & kOneOne;
          v.z = __byte_perm(eq, 0u, 0x2222u) & kOneOne;
          v.w = __byte_perm(eq, 0u, 0x3333u) & kOneOne;
          const uint32_t off = my_row_off[kk] + (uint32_t)(q4 >> 1) * (uint32_t)(Nm * 32) + (uint32_t)(q4 & 1) * 128u;
          *reinterpret_cast<uint4*>(hs + off) = v;
        }
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        if (!mbar_wait(&bar_v[s], ph_v[s])) {
          atomicOr(a.status, kStatusTimeout);
          *s_abort = 1;
        } else {
          fence_after_sync();
          const uint32_t va = smem_addr(sV + s * kShChunkBytes), ha = smem_addr(hs);
#pragma unroll
          for (int ks = 0; ks < kShKSteps; ++ks) {
            const uint64_t dv = smem_desc(va + (uint32_t)ks * (kShRows * 32u));
            const uint32_t acc = (ch > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
            for (int op = 0; op < 2; ++op) {
              const uint64_t dh = smem_desc(ha + (uint32_t)op * (uint32_t)(Nm * kShK * 2) + (uint32_t)ks * (uint32_t)(Nm * 32));
              mma_f16(tmem + (uint32_t)op * 256u, dv, dh, idesc, acc);
            }
          }
          mma_commit(&bar_mma[s]);
        }
      }
      ph_v[s] ^= 1u;
      pend[s] = true;
      __syncthreads();
      if (*s_abort) {
        abort = true;
        break;
      }
    }
    // drain this item's MMAs
    bool fail = false;
    for (int s = 0; s < 2; ++s)
      if (pend[s]) {
        fail |= !mbar_wait(&bar_mma[s], ph_mma[s]);
        ph_mma[s] ^= 1u;
        pend[s] = false;
      }
    if (__syncthreads_or(fail)) abort = true;
    if (abort) break;
    fence_after_sync();

    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 of accumulator w / 4
    const int quarter = warp & 3, op = warp >> 2;
    const int row = quarter * 32 + lane;
    const int64_t c = g * kShCurves + (row >> 1);
    const bool even = (row & 1) == 0;
    const bool cvalid = c < a.ncurves;
    const float sa = cvalid ? a.inv_scale[2 * c] : 0.f, sw = cvalid ? a.inv_scale[2 * c + 1] : 0.f;
    const bool cbad = cvalid && a.curve_bad[c];
    float acc = 0.f;
    int m = 0, jl = 0;
    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)op * 256u;
    for (int c0 = 0; c0 < rows_used; c0 += 8) {
      uint32_t v[8];
      if (nch > 0) {
        tmem_ld8(tbase + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = 0u;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (c0 + u >= rows_used) break;
        const float val = __uint_as_float(v[u]);
        const float other = __shfl_xor_sync(0xffffffffu, val, 1);
        if (even) {
          const float A = val * sa, B = other * sw;
          const float den = B + cal;
          acc += den > 0.f ? (A * A) / den : 0.f;
        }
        if (++m == M) {
          const int64_t fi = f0 + (int64_t)op * fpm + jl;
          if (even && cvalid && fi < F) {
            const float S = cbad ? __int_as_float(0x7fc00000) : acc;
            if (a.S32) a.S32[c * F + fi] = S;
            if (a.S_out) a.S_out[c * F + fi] = (double)S;
          }
          acc = 0.f;
          m = 0;
          ++jl;
        }
      }
    }
    fence_before_sync();
    __syncthreads();
  }
  // teardown: nothing of this CTA may still be in flight when TMEM is freed
  for (int s = 0; s < 2; ++s)
    if (pend[s]) {
      if (!mbar_wait(&bar_mma[s], ph_mma[s])) atomicOr(a.status, kStatusTimeout);
      pend[s] = false;
    }
  if (abort && tid == 0) atomicOr(a.status, kStatusTimeout);
  fence_before_sync();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kShTmemCols) : "memory");
}

// ---------------------------------------------------------------- top-k
// One block per curve over its dense FP32 periodogram: k rounds of a block
// arg-max among peaks ranked strictly after the previous pick.
constexpr int kShTopkThreads = 512;

__global__ void __launch_bounds__(kShTopkThreads) shared_topk_kernel(const SharedArgs a) {
  __shared__ float ws[32];
  __shared__ int wi[32];
  const int64_t c = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t F = a.nfreq;
  const float* S = a.S32 + c * F;
  const bool grid_bad = (*(volatile unsigned*)a.status & kStatusGrid) != 0u;
  const bool bad = grid_bad || a.curve_bad[c];
  int32_t* oi = a.topk_idx + c * a.k;
  float* os = a.topk_S + c * a.k;
  float ps = INFINITY;
  int pi = -1;
  for (int q = 0; q < a.k; ++q) {
    float bs = -INFINITY;
    int bi = -1;
    if (!bad) {
      for (int64_t e = tid; e < F; e += kShTopkThreads) {
        const float s = S[e];
        bool peak = true;
        if (!a.peak_raw) {
          const float l = (e > 0) ? S[e - 1] : -INFINITY;
          const float r = (e + 1 < F) ? S[e + 1] : -INFINITY;
          peak = (e == 0) ? (F == 1 || s >= r) : (e + 1 == F ? s > l : (s > l && s >= r));
        }
        if (!peak) continue;
        const bool after = (q == 0) || ranks_before((double)ps, pi, (double)s, (int)e);
        if (after && (bi < 0 || ranks_before((double)s, (int)e, (double)bs, bi))) {
          bs = s;
          bi = (int)e;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os_ = __shfl_xor_sync(0xffffffffu, bs, o);
      const int oi_ = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oi_ >= 0 && (bi < 0 || ranks_before((double)os_, oi_, (double)bs, bi))) {
        bs = os_;
        bi = oi_;
      }
    }
    if (lane == 0) {
      ws[warp] = bs;
      wi[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      bs = lane < (kShTopkThreads >> 5) ? ws[lane] : -INFINITY;
      bi = lane < (kShTopkThreads >> 5) ? wi[lane] : -1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float os_ = __shfl_xor_sync(0xffffffffu, bs, o);
        const int oi_ = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi_ >= 0 && (bi < 0 || ranks_before((double)os_, oi_, (double)bs, bi))) {
          bs = os_;
          bi = oi_;
        }
      }
      if (lane == 0) {
        oi[q] = bi;
        os[q] = bi >= 0 ? bs : __int_as_float(0x7fc00000);
        ws[0] = bs;
        wi[0] = bi;
      }
    }
    __syncthreads();
    ps = ws[0];
    pi = wi[0];
    __syncthreads();
    if (pi < 0) {
      for (int r = q + 1 + tid; r < a.k; r += kShTopkThreads) {
        oi[r] = -1;
        os[r] = __int_as_float(0x7fc00000);
      }
      break;
    }
  }
}

}  // namespace

size_t shared_image_bytes(int64_t ncurves, int64_t n) {
  const int64_t groups = (ncurves + kShCurves - 1) / kShCurves;
  const int64_t nch = (n + kShObs - 1) / kShObs;
  return (size_t)groups * (size_t)nch * kShChunkBytes;
}

int shared_curves_per_group() { return kShCurves; }

// Frequencies per accumulator and the MMA's N for M bins (0 if M is too large).
int shared_freqs_per_mma(int M, int* n_mma) {
  if (M < 1 || M > kShNMax) return 0;
  const int fpm = kShNMax / M;
  *n_mma = ((fpm * M + 15) / 16) * 16;
  return fpm;
}

cudaError_t shared_init_attributes() {
  return cudaFuncSetAttribute(shared_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

size_t shared_smem_bytes() { return kSmemBytes; }

cudaError_t launch_shared(const SharedArgs& a, int nsm, cudaStream_t st) {
  const int64_t slots = a.ngroups * kShCurves;
  if (slots <= 0) return cudaSuccess;
  shared_prep_kernel<<<(unsigned)slots, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t items = a.ngroups * a.npass;
  if (items > 0) {
    const int grid = (int)(items < nsm ? items : nsm);
    if (a.timing_start) cudaEventRecord(a.timing_start, st);
    shared_mma_kernel<<<grid, kShThreads, kSmemBytes, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.timing_stop) cudaEventRecord(a.timing_stop, st);
  }
  if (a.k > 0 && a.ncurves > 0) {
    shared_topk_kernel<<<(unsigned)a.ncurves, kShTopkThreads, 0, st>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace fpw
