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
constexpr int kShThreads = 576;  // 16 builder/epilogue warps + 2 issuer warps
constexpr int kShNMax = 256;                    // MMA N limit (M = 128)
constexpr int kShMaxFpm = 64;                   // frequencies per accumulator, at most
constexpr int kShHOperandMax = kShNMax * kShK * 2;   // one H operand of a chunk: 32 KB
constexpr int kShHSlotBytes = 2 * kShHOperandMax;    // two H operands (two accumulators)
constexpr int kShTmemCols = 512;
constexpr unsigned kOneOne = 0x3C003C00u;       // two fp16 1.0
constexpr long long kWaitClocks = 4000000000LL; // default wait limit, ~2 s at 2 GHz
// A waiting thread is suspended in mbarrier.try_wait until the phase completes
// or this many nanoseconds pass (so waiting warps do not take issue slots).
constexpr uint32_t kSuspendNs = 20000u;
constexpr int kMaxPassFreqs = 2 * kShMaxFpm;
constexpr int kMaxPairs = kMaxPassFreqs * kShObs;
constexpr int kShVSlots = 4;                    // V chunks in flight: loads run two chunks ahead
constexpr int kShStage = 1024;                  // observations staged at a time (t, anchor P, step D)
constexpr int kShStageChunks = kShStage / kShObs;

// Shared-memory carve-up (bytes).
constexpr int kOffV = 0;                                   // V chunks: 4 x 16 KB
constexpr int kOffH = kOffV + kShVSlots * kShChunkBytes;   // H chunks: 2 x 64 KB
constexpr int kOffOld = kOffH + 2 * kShHSlotBytes;         // bin of every (frequency, observation) pair in H, per slot
constexpr int kOffF = kOffOld + 2 * kMaxPairs;             // the pass's frequencies (binary64)
constexpr int kOffStage = kOffF + kMaxPassFreqs * 8;       // t, P, D of kShStage observations
constexpr int kOffPart = kOffStage + 3 * kShStage * 8;    // epilogue: partial S of a frequency split between warps
constexpr int kOffBar = kOffPart + 2 * 128 * 4;
constexpr int kSmemBytes = kOffBar + 128;

// Byte offset of element (row r, k-entry q) of a K-major, unswizzled operand
// with R rows and kShK columns: one 16-column k-step after another; inside a
// k-step, 8-row x 16-byte core matrices, the two of a row group adjacent (the
// K-direction stride, 128 B) and row groups 256 B apart.
__host__ __device__ __forceinline__ uint32_t km_off(uint32_t r, uint32_t q, uint32_t R) {
  return (q >> 4) * (R * 32u) + (r >> 3) * 256u + ((q >> 3) & 1u) * 128u + (r & 7u) * 16u + (q & 7u) * 2u;
}

// Approximate reciprocal (one special-function instruction, relative error
// about 2^-23), subnormal inputs and results flushed to zero: the epilogue
// drops denominators below FLT_MIN, and a reciprocal that flushes (a
// denominator above 2^126) leaves a term far below the absolute tolerance.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
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

// Bounded wait for completion of phase `parity` of an mbarrier.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitClocks) return false;
  }
}

// mbarrier wait of the chunk pipeline: gives up after `limit` clocks or when
// another role of the CTA set *abort; `suspend_ns` is the longest time one
// try_wait may suspend the thread.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort, long long limit,
                                             uint32_t suspend_ns) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(suspend_ns)
        : "memory");
    if (done) return true;
    if (*abort || clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void mbar_init_n(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Named barrier among the builder warps only (the issuer warp never joins).
__device__ __forceinline__ void builders_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

__device__ __forceinline__ bool builders_or(bool v, int nthreads) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(nthreads)
      : "memory");
  return r != 0u;
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

// tcgen05.ld of 8 columns without the wait; the registers are valid only after
// tmem_wait_ld8 on the same array, which names them as operands so that no
// use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld8_issue(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld8(uint32_t (&v)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])
               :
               : "memory");
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

// ---------------------------------------------------------------- phase steps
// Per observation: the 64-bit phase step D_i = frac(t_i df) for the grid's
// mean spacing df, and max |t| (for the grid-linearity bound).
__global__ void shared_steps_kernel(const SharedArgs a) {
  const int64_t F = a.nfreq;
  const double df = (F > 1) ? (a.freqs[F - 1] - a.freqs[0]) / (double)(F - 1) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double t = a.t[i];
    const bool ok = isfinite(t) && isfinite(df);
    a.step[i] = ok ? phase_fixed64(t, df) : 0ull;
    if (ok) atomicMax(a.tmax_bits, (unsigned long long)__double_as_longlong(fabs(t)));
  }
}

// ---------------------------------------------------------------- MMA kernel
// Warp-specialised pipeline over this CTA's stream of chunks (32 observations
// of one item each; gc counts them across items):
//  * builder warps (0-14): for chunk gc, wait until the MMAs of gc - 2 have
//    released H slot gc & 1 (mbarrier `empty`), then each (frequency,
//    observation) pair clears its previous one in that slot and sets its new
//    one (pairs own disjoint 4-byte words; phases step from staged anchors,
//    Phi = P_i + j D_i, when the pass lies on the linear grid, else exact
//    anchors per pair); each warp then arrives on `full`. At an item's end
//    warps 0-7 read the accumulators (after `acc`) and arrive on `tfree`.
//  * issuer warp (15, one lane): waits for `full`, starts the bulk copy of the
//    V chunk two chunks ahead (its slot was last read by the MMAs of gc - 2,
//    complete once `full` of gc has completed), waits for V of gc (and, on an
//    item's first chunk, for `tfree`), issues the 2 x 4 MMAs and commits them
//    to `empty` (and to `acc` after an item's last chunk).
// No block-wide barrier inside the loop; every wait is bounded and gives up
// when another role has set the abort flag.
constexpr int kShBuilderWarps = 16;
constexpr int kShBuilders = kShBuilderWarps * 32;
constexpr int kShIssuers = kShThreads / 32 - kShBuilderWarps;  // one per accumulator

__global__ void __launch_bounds__(kShThreads, 1) shared_mma_kernel(const SharedArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sV = smem + kOffV;
  unsigned char* sH = smem + kOffH;
  uint8_t* sOld = smem + kOffOld;
  double* sF = reinterpret_cast<double*>(smem + kOffF);
  double* sT = reinterpret_cast<double*>(smem + kOffStage);
  unsigned long long* sP = reinterpret_cast<unsigned long long*>(sT + kShStage);
  unsigned long long* sD = sP + kShStage;
  uint64_t* bar_full = reinterpret_cast<uint64_t*>(smem + kOffBar);  // [2]
  uint64_t* bar_empty = bar_full + 2;                                 // [2]
  uint64_t* bar_v = bar_empty + 2;                                    // [kShVSlots]
  uint64_t* bar_acc = bar_v + kShVSlots;
  uint64_t* bar_tfree = bar_acc + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar_tfree + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int M = a.M, fpm = a.fpm, Nm = a.n_mma, FP = 2 * fpm, rows_used = fpm * M;
  const int npairs = FP * kShObs;
  const int64_t F = a.nfreq, n = a.n, nch = a.nchunks;
  const bool resident = n <= kShStage;
  const bool grid_bad = (*(volatile unsigned*)a.status & kStatusGrid) != 0u;
  const int64_t items = grid_bad ? 0 : a.ngroups * a.npass;
  const int64_t my_items = (int64_t)blockIdx.x < items ? (items - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const float cal = (float)a.inv_alpha2;
  const double df = (F > 1) ? (a.freqs[F - 1] - a.freqs[0]) / (double)(F - 1) : 0.0;
  const double tmax = __longlong_as_double((long long)*a.tmax_bits);
  const uint32_t op_bytes = (uint32_t)(Nm * kShK * 2);  // one H operand
  // byte offset of this lane's observation (hi, lo) word inside a row of H
  const uint32_t lane_off = (uint32_t)(lane >> 3) * (uint32_t)(Nm * 32) + (uint32_t)((lane >> 2) & 1) * 128u +
                            (uint32_t)(lane & 3) * 4u;

  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      mbar_init_n(&bar_full[q], kShBuilderWarps);
      mbar_init_n(&bar_empty[q], kShIssuers);
    }
    for (int v = 0; v < kShVSlots; ++v) mbar_init_n(&bar_v[v], 1);
    mbar_init_n(bar_acc, kShIssuers);
    mbar_init_n(bar_tfree, kShBuilderWarps);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(kShTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // H starts as all pairs in bin 0 (rows beyond fpm * M stay zero for good)
  for (int e = tid; e < 2 * kShHSlotBytes / 16; e += kShThreads)
    reinterpret_cast<uint4*>(sH)[e] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int e = tid; e < npairs; e += kShThreads) {
    const int j = e >> 5;
    const int op = j >= fpm ? 1 : 0;
    const uint32_t r = (uint32_t)((j - op * fpm) * M);
    const uint32_t w = lane_off + (uint32_t)op * op_bytes + (r >> 3) * 256u + (r & 7u) * 16u;
    for (int q = 0; q < 2; ++q) {
      *reinterpret_cast<uint32_t*>(sH + q * kShHSlotBytes + w) = kOneOne;
      sOld[q * kMaxPairs + e] = 0;
    }
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  bool fail = false;
  // limit of the pipeline's waits (the drain after a failure keeps the
  // default); a limit far below one suspension also stops each try_wait from
  // suspending, so that a wait whose phase is not complete gives up at once
  const long long wait_limit = a.wait_clocks > 0 ? a.wait_clocks : kWaitClocks;
  const uint32_t suspend_ns = wait_limit < 100000 ? 0u : kSuspendNs;

  if (warp >= kShBuilderWarps) {
    // ------------------------------------------------------------ issuers: warp 16 drives accumulator 0 and
    // the V loads, warp 17 accumulator 1; both commit to `empty` and `acc` (count 2)
    const int iop = warp - kShBuilderWarps;
    if (lane == 0 && my_items > 0 && nch > 0) {
      const uint32_t idesc = mma_idesc(kShRows, Nm);
      // descriptors of chunk operands: a base descriptor plus the byte offset / 16
      // in the start-address field (all offsets stay inside shared memory)
      const uint64_t dv0 = smem_desc(smem_addr(sV)), dh0 = smem_desc(smem_addr(sH));
      const int64_t total = my_items * nch;
      // the V-load cursor (item lk of this CTA, chunk lch) runs two chunks ahead
      // of the MMA cursor; both advance incrementally (no 64-bit division per chunk)
      int64_t lk = 0, lch = 0;
      const unsigned char* limg = a.image + (size_t)(blockIdx.x / a.npass) * (size_t)nch * kShChunkBytes;
      auto load_next = [&](int slot) {
        bulk_load(sV + slot * kShChunkBytes, limg + (size_t)lch * kShChunkBytes, kShChunkBytes, &bar_v[slot]);
        if (++lch == nch) {
          lch = 0;
          ++lk;
          const int64_t it = blockIdx.x + lk * gridDim.x;
          limg = a.image + (size_t)(it / a.npass) * (size_t)nch * kShChunkBytes;
        }
      };
      if (iop == 0)
        for (int64_t c = 0; c < 2 && c < total; ++c) load_next((int)c);
      // per-slot phase parities and flags as bit masks in registers (a
      // run-time-indexed array would live in local memory)
      uint32_t ph_full = 0u, ph_v = 0u, ph_tfree = 0u;
      uint32_t commits0 = 0u, commits1 = 0u;
      uint32_t v_out = iop == 0 ? ((total > 0 ? 1u : 0u) | (total > 1 ? 2u : 0u)) : 0u;  // own loads in flight
      int64_t ch = 0;
      for (int64_t gc = 0; gc < total && !fail; ++gc, ch = (ch + 1 == nch) ? 0 : ch + 1) {
        const int s = (int)(gc & 1), vs = (int)(gc & (kShVSlots - 1));
        if (!mbar_wait_ab(&bar_full[s], (ph_full >> s) & 1u, s_abort, wait_limit, suspend_ns)) { fail = true; break; }
        ph_full ^= 1u << s;
        if (iop == 0 && gc + 2 < total) {  // its slot was last read by the MMAs of gc - 2, done before `full` of gc
          const int v2 = (int)((gc + 2) & (kShVSlots - 1));
          load_next(v2);
          v_out |= 1u << v2;
        }
        if (!mbar_wait_ab(&bar_v[vs], (ph_v >> vs) & 1u, s_abort, wait_limit, suspend_ns)) { fail = true; break; }
        ph_v ^= 1u << vs;
        v_out &= ~(1u << vs);
        if (ch == 0 && gc > 0) {  // the previous item's accumulators have been read
          if (!mbar_wait_ab(bar_tfree, ph_tfree, s_abort, wait_limit, suspend_ns)) { fail = true; break; }
          ph_tfree ^= 1u;
        }
        fence_after_sync();
        const uint64_t dvs = dv0 + (uint64_t)((vs * kShChunkBytes) >> 4);
        const uint64_t dhs = dh0 + (uint64_t)((s * kShHSlotBytes + iop * (int)op_bytes) >> 4);
#pragma unroll
        for (int ks = 0; ks < kShKSteps; ++ks) {
          const uint32_t acc = (ch > 0 || ks > 0) ? 1u : 0u;
          mma_f16(tmem + (uint32_t)iop * 256u, dvs + (uint64_t)((ks * kShRows * 32) >> 4),
                  dhs + (uint64_t)(((uint32_t)ks * (uint32_t)(Nm * 32)) >> 4), idesc, acc);
        }
        mma_commit(&bar_empty[s]);
        if (s == 0) ++commits0; else ++commits1;
        if (ch == nch - 1) mma_commit(bar_acc);
      }
      if (fail) {
        *s_abort = 1;
        atomicOr(a.status, kStatusTimeout);
        // nothing may be in flight when the CTA frees TMEM and exits: bounded
        // waits for the last commit of each slot and for outstanding V loads
        for (int q = 0; q < 2; ++q)
          if ((q == 0 ? commits0 : commits1) > 0u) mbar_wait(&bar_empty[q], ((q == 0 ? commits0 : commits1) - 1u) & 1u);
        for (int v = 0; v < kShVSlots; ++v)
          if ((v_out >> v) & 1u) mbar_wait(&bar_v[v], (ph_v >> v) & 1u);
      }
    }
  } else {
    // ------------------------------------------------------------ builders (+ epilogue in warps 0-7)
    // Every builder runs the same loops to the end and passes every named
    // barrier even after a failure (it then skips the work), so no builder
    // can wait at a barrier for one that left; failure decisions are made
    // warp-uniform before any warp-collective instruction.
    uint32_t ph_empty = 0u, ph_acc = 0u;  // per-slot parities as bits
    bool staged = false;
    int64_t gc = 0;
    for (int64_t k = 0; k < my_items; ++k) {
      const int64_t item = blockIdx.x + k * gridDim.x;
      const int64_t g = item / a.npass, p = item % a.npass;
      const int64_t f0 = p * FP;
      const double fa = a.freqs[f0];
      if (k > 0) builders_sync(kShBuilders);  // every builder is done with the previous item's sF and stage
      bool nonlin = false;
      for (int j = tid; j < FP; j += kShBuilders) {
        const int64_t fi = f0 + j;
        const double f = fi < F ? a.freqs[fi] : 0.0;
        sF[j] = f;
        if (fi < F && fabs(f - fma((double)j, df, fa)) * tmax > kGridTolCycles) nonlin = true;
      }
      const bool lin = !builders_or(nonlin, kShBuilders);
      for (int64_t ch = 0; ch < nch; ++ch, ++gc) {
        const int s = (int)(gc & 1);
        if (ch % kShStageChunks == 0) {  // stage a block of observations (same thread per entry throughout)
          if (ch > 0) builders_sync(kShBuilders);
          const int64_t o0 = ch * kShObs;
          for (int i = tid; i < kShStage; i += kShBuilders) {
            const int64_t oi = o0 + i;
            if (!resident || !staged) {
              sT[i] = oi < n ? a.t[oi] : 0.0;
              sD[i] = oi < n ? a.step[oi] : 0ull;
            }
            sP[i] = phase_fixed64(sT[i], fa);
          }
          staged = true;
          builders_sync(kShBuilders);
        }
        if (!fail && gc >= 2) {  // the MMAs of gc - 2 read H slot s
          fail = !mbar_wait_ab(&bar_empty[s], (ph_empty >> s) & 1u, s_abort, wait_limit, suspend_ns);
          ph_empty ^= 1u << s;
        }
        fail = __any_sync(0xffffffffu, fail);
        if (fail && lane == 0) *s_abort = 1;  // the other roles stop waiting
        if (!fail) {
          unsigned char* hs = sH + s * kShHSlotBytes;
          uint8_t* old = sOld + s * kMaxPairs;
          const int ib = (int)(ch % kShStageChunks) * kShObs + lane;
          const bool obs_ok = ch * kShObs + lane < n;
          const unsigned long long P = sP[ib], D = sD[ib];
          const double tl = sT[ib];
          // pair e = (frequency e / 32, this lane's observation): clear its
          // previous one and set its new one; two pairs at a time, both bins
          // and both previous bins read before any store (the pairs' rows are
          // disjoint)
          auto put = [&](int e, unsigned m, unsigned mo) {
            const int j = e >> 5;  // warp-uniform
            const int op = j >= fpm ? 1 : 0;
            const uint32_t r0 = (uint32_t)((j - op * fpm) * M);
            const uint32_t base = lane_off + (uint32_t)op * op_bytes;
            const uint32_t ro = r0 + mo, rn = r0 + m;
            *reinterpret_cast<uint32_t*>(hs + base + (ro >> 3) * 256u + (ro & 7u) * 16u) = 0u;
            *reinterpret_cast<uint32_t*>(hs + base + (rn >> 3) * 256u + (rn & 7u) * 16u) = kOneOne;
            old[e] = (uint8_t)m;
          };
          if (lin) {
            for (int e = tid; e < npairs; e += 2 * kShBuilders) {
              const int e2 = e + kShBuilders;
              const bool two = e2 < npairs;  // warp-uniform
              const int ja = e >> 5, jb = e2 >> 5;
              const unsigned ma = (obs_ok && f0 + ja < F) ? bin_of_phase(P + (unsigned long long)ja * D, (unsigned)M) : 0u;
              const unsigned mb =
                  (two && obs_ok && f0 + jb < F) ? bin_of_phase(P + (unsigned long long)jb * D, (unsigned)M) : 0u;
              const unsigned oa = old[e], ob = two ? old[e2] : 0u;
              put(e, ma, oa);
              if (two) put(e2, mb, ob);
            }
          } else {
            for (int e = tid; e < npairs; e += kShBuilders) {
              const int j = e >> 5;
              const unsigned m = (obs_ok && f0 + j < F) ? bin_of_phase(phase_fixed64(tl, sF[j]), (unsigned)M) : 0u;
              put(e, m, old[e]);
            }
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bar_full[s]);
        }
      }
      // epilogue: all builder warps. Warp w reads TMEM lanes 32 (w % 4) .. + 31
      // of accumulator (w / 4) % 2, columns [0, split) for w < 8 and
      // [split, fpm M) above (split a multiple of 8 near the middle); the
      // partial sum of a frequency that straddles the split is handed over
      // through shared memory.
      float* sPart = reinterpret_cast<float*>(smem + kOffPart);
      if (!fail && nch > 0) {
        fail = !mbar_wait_ab(bar_acc, ph_acc, s_abort, wait_limit, suspend_ns);
        fence_after_sync();
      }
      fail = __any_sync(0xffffffffu, fail);
      if (fail && lane == 0) *s_abort = 1;
      const int quarter = warp & 3, op = (warp >> 2) & 1, half = warp >> 3;
      const int row = quarter * 32 + lane;
      const int64_t c = g * kShCurves + (row >> 1);
      const bool cvalid = c < a.ncurves;
      const int split = ((rows_used + 15) >> 4) << 3;
      const int js = split / M;                          // frequency holding column `split`
      const bool straddle = split < rows_used && split % M != 0;
      const int64_t fbase = f0 + (int64_t)op * fpm;
      const int jmax = (int)((F - fbase) < fpm ? (F - fbase) : fpm);
      const bool cbad = cvalid && a.curve_bad[c];
      // both lanes of a pair store the pair's sum to the same address
      // (one transaction, no divergent branch before the next shuffle); lanes
      // of padding curves write into a scratch area instead
      float* const s32 = a.S32 ? (cvalid ? a.S32 + c * F + fbase : a.scratch32 + lane * kShMaxFpm) : nullptr;
      double* const s64 = a.S_out ? (cvalid ? a.S_out + c * F + fbase : a.scratch64 + lane * kShMaxFpm) : nullptr;
      const float nan = __int_as_float(0x7fc00000);
      // this lane's part of the running frequency sum; the two lanes of a
      // curve's pair add up to the sum
      float acc = 0.f;
      if (!fail) {
        // lanes 2c and 2c + 1 hold the A and B rows of curve c. For M >= 8 the
        // pair splits each block of 8 columns: one shuffle per two columns gives
        // the even lane B of an even column and the odd lane A of an odd one, so
        // each lane forms the terms A^2 / (B + 1/alpha^2) of its own columns, and
        // a block holds at most one frequency end. Below 8 bins the even lane
        // forms every term.
        const float sa = cvalid ? a.inv_scale[2 * c] : 0.f, sw = cvalid ? a.inv_scale[2 * c + 1] : 0.f;
        const int cb = half == 0 ? 0 : split, ce = half == 0 ? split : rows_used;
        const int par = lane & 1;
        int jl = cb / M;
        int fend = (jl + 1) * M;  // the column where frequency jl ends (warp-uniform)
        auto emit = [&](float S) {  // frequency jl complete
          if (half == 1 && straddle && jl == js) {
            sPart[op * 128 + row] = S;  // the second part of the straddling frequency
          } else if (jl < jmax) {
            if (s32) s32[jl] = cbad ? nan : S;
            if (s64) s64[jl] = cbad ? (double)nan : (double)S;
          }
        };
        const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)op * 256u;
        // 8 columns per step; the next step's TMEM load is in flight while
        // this step's columns are reduced
        uint32_t nx[8];
        if (nch > 0 && cb < ce) tmem_ld8_issue(tbase + (uint32_t)cb, nx);
        for (int c0 = cb; c0 < ce; c0 += 8) {
          uint32_t v[8];
          if (nch > 0) {
            tmem_wait_ld8(nx);
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = nx[u];
            if (c0 + 8 < ce) tmem_ld8_issue(tbase + (uint32_t)(c0 + 8), nx);
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = 0u;
          }
          if (M >= 8) {
            float lo = 0.f, hi = 0.f;  // this lane's terms before / after the frequency end
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float ev = __uint_as_float(v[2 * q]), od = __uint_as_float(v[2 * q + 1]);
              const float recv = __shfl_xor_sync(0xffffffffu, par ? ev : od, 1);
              const float A = (par ? recv : ev) * sa;
              const float den = (par ? od : recv) * sw + cal;
              const int col = c0 + 2 * q + par;
              const float term = (den >= 1.17549435e-38f && col < ce) ? (A * A) * rcp_approx(den) : 0.f;
              lo += col < fend ? term : 0.f;
              hi += col < fend ? 0.f : term;
            }
            acc += lo;
            if (fend <= c0 + 8 && fend <= ce) {
              emit(acc + __shfl_xor_sync(0xffffffffu, acc, 1));
              acc = hi;
              ++jl;
              fend += M;
            }
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const float val = __uint_as_float(v[u]);
              const float other = __shfl_xor_sync(0xffffffffu, val, 1);
              const float A = val * sa;
              const float den = other * sw + cal;
              acc += (par == 0 && den >= 1.17549435e-38f && c0 + u < ce) ? (A * A) * rcp_approx(den) : 0.f;
              if (c0 + u < ce && c0 + u + 1 == fend) {  // warp-uniform
                emit(acc + __shfl_xor_sync(0xffffffffu, acc, 1));
                acc = 0.f;
                ++jl;
                fend += M;
              }
            }
          }
        }
      }
      fence_before_sync();
      builders_sync(kShBuilders);  // partial sums visible; every TMEM read of this item done
      if (!fail && half == 0 && straddle && js < jmax) {
        const float S = acc + __shfl_xor_sync(0xffffffffu, acc, 1) + sPart[op * 128 + (row & ~1)];
        if (s32) s32[js] = cbad ? nan : S;
        if (s64) s64[js] = cbad ? (double)nan : (double)S;
      }
      if (!fail && nch > 0 && lane == 0) mbar_arrive(bar_tfree);
      ph_acc ^= 1u;
    }
    if (fail) {
      *s_abort = 1;
      atomicOr(a.status, kStatusTimeout);
    }
  }
  // teardown: on success the last epilogue waited for `acc`, which covers
  // every MMA, and every V load was waited for; after a failure the issuer
  // drained its own work above
  fence_before_sync();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kShTmemCols) : "memory");
}

// ---------------------------------------------------------------- top-k
// One block per curve over its dense FP32 periodogram: k rounds of a block
// arg-max among peaks ranked strictly after the previous pick.
constexpr int kShTopkThreads = 512;

__global__ void __launch_bounds__(kShTopkThreads) dense_topk32_kernel(const DenseTopk32Args a) {
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
  const int fpm = kShNMax / M < kShMaxFpm ? kShNMax / M : kShMaxFpm;
  *n_mma = ((fpm * M + 15) / 16) * 16;
  return fpm;
}

cudaError_t launch_dense_topk32(const DenseTopk32Args& t, int64_t ncurves, cudaStream_t st) {
  if (t.k <= 0 || ncurves <= 0) return cudaSuccess;
  dense_topk32_kernel<<<(unsigned)ncurves, kShTopkThreads, 0, st>>>(t);
  return cudaGetLastError();
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
  e = cudaMemsetAsync(a.tmax_bits, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (a.n > 0) {
    const int64_t blocks = (a.n + 255) / 256;
    shared_steps_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
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
