// fpw_periodogram_batch_noalloc: the batched periodogram for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or allocator, plugins whose host forbids device
// allocation after start-up, and real-time pipelines that must not risk an
// allocation failure or an implicit device synchronization in the middle of a
// run. This entry point allocates nothing. Its scratch memory (weights, work
// list, per-curve flags, peak candidates, status words) lives in one
// file-scope __device__ array of kScratchBytes, which every GPU that loads
// the library holds until the process exits. The caller still provides the
// inputs and outputs.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in). The first call on each device, with that device
// current, looks up the device address with cudaGetSymbolAddress and keeps it;
// make that first call before any stream capture. Every call shares the one
// array and overwrites it, so calls whose work overlaps on the GPU (different
// streams or host threads) race: serialize them.
#include <mutex>

#include "fpw_internal.cuh"

namespace fpw {
namespace {

// Largest scratch the entry point may use: about 4 million observations of
// FP32 weights plus the work list and candidates of their curves.
constexpr size_t kScratchBytes = (size_t)32 << 20;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSetup {
  bool done = false;
  unsigned char* scratch = nullptr;  // device address of g_scratch on this device
  int nsm = 0;
  int smem_optin = 0;
  int smem_per_sm = 0;
};

std::mutex g_setup_mu;
DeviceSetup g_setup[64];

// Work list: one item per curve, ordered by decreasing size class (a counting
// sort on floor(log2 n) + 1 in the scratch array), so that the persistent
// kernel starts the longest curves first. Within a class the order is
// whatever the atomics give; it changes no result, only the schedule.
constexpr int kSizeClasses = 64;

__device__ __forceinline__ int size_class(const int64_t* offsets, int64_t c) {
  const int64_t n = offsets[c + 1] - offsets[c];
  return n > 0 ? __clzll((long long)n) : 63;  // larger n, smaller class
}

__global__ void noalloc_count_kernel(const int64_t* offsets, int64_t C, unsigned* hist, int32_t* cand_base) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= C; c += (int64_t)gridDim.x * blockDim.x) {
    cand_base[c] = (int32_t)c;
    if (c < C) atomicAdd(&hist[size_class(offsets, c)], 1u);
  }
}

__global__ void noalloc_scan_kernel(unsigned* hist) {  // one thread: exclusive prefix sums, in place
  unsigned run = 0;
  for (int q = 0; q < kSizeClasses; ++q) {
    const unsigned h = hist[q];
    hist[q] = run;
    run += h;
  }
}

__global__ void noalloc_items_kernel(const int64_t* offsets, int64_t C, int64_t F, unsigned* cursor, WorkItem* items) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
    const unsigned pos = atomicAdd(&cursor[size_class(offsets, c)], 1u);
    WorkItem w;
    w.curve = (int32_t)c;
    w.f_lo = 0;
    w.f_hi = (int32_t)F;
    w.slot = (int32_t)c;
    items[pos] = w;
  }
}

// offsets[0] = 0, non-decreasing, total <= 2^40; `prev` carries the last
// offset of the previous chunk (-1 for the first).
bool offsets_chunk_ok(const int64_t* o, int64_t cnt, int64_t& prev) {
  for (int64_t q = 0; q < cnt; ++q) {
    if (prev < 0 ? o[q] != 0 : o[q] < prev) return false;
    if (o[q] > ((int64_t)1 << 40)) return false;
    prev = o[q];
  }
  return true;
}

int setup_device(int dev, DeviceSetup** out) {
  if (dev < 0 || dev >= 64) return FPW_EINVAL;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.done) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) return FPW_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return FPW_ECUDA;
    if (tile_init_attributes((int)prop.sharedMemPerBlockOptin) != cudaSuccess) return FPW_ECUDA;
    s.scratch = static_cast<unsigned char*>(p);
    s.nsm = prop.multiProcessorCount;
    s.smem_optin = (int)prop.sharedMemPerBlockOptin;
    s.smem_per_sm = (int)prop.sharedMemPerMultiprocessor;
    s.done = true;
  }
  *out = &s;
  return FPW_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace fpw

using namespace fpw;

extern "C" FPW_API int fpw_periodogram_batch_noalloc(void* stream, const fpw_params* params, const int64_t* offsets,
                                                     const int64_t* offsets_host, int64_t ncurves, const double* t,
                                                     const double* x, const double* sigma, const double* freqs,
                                                     int64_t nfreq, int M, int k, int32_t* topk_idx, float* topk_S) {
  if (ncurves < 0 || nfreq < 0 || M < 1 || k < 0 || k > FPW_MAX_TOPK) return FPW_EINVAL;
  if (ncurves == 0) return FPW_OK;
  if (!offsets || nfreq == 0 || !freqs || (k > 0 && (!topk_idx || !topk_S))) return FPW_EINVAL;
  if (nfreq > ((int64_t)1 << 31) - 1024 || ncurves > ((int64_t)1 << 31) - 1) return FPW_EINVAL;
  fpw_params p;
  fpw_params_default(&p);
  if (params) p = *params;
  if (!(p.inv_alpha2 >= 0.0) || p.inv_alpha2 > 1e300 || p.K < 1) return FPW_EINVAL;
  if (p.phase_mode != FPW_PHASE_FIXED64 && p.phase_mode != FPW_PHASE_FP32) return FPW_ENOTSUP;
  if (p.accum != FPW_ACCUM_FP32 && p.accum != FPW_ACCUM_FP64 && p.accum != FPW_ACCUM_FP32_COMP) return FPW_EINVAL;
  if (p.threads != 0 && (p.threads < 32 || p.threads > 512 || p.threads % 32 != 0)) return FPW_EINVAL;
  if (p.freqs_per_thread != 0 && !tile_supported_R(p.freqs_per_thread)) return FPW_EINVAL;
  if (p.obs_chunk != 0 && p.obs_chunk < 32) return FPW_EINVAL;
  if (p.items_per_slot < 0) return FPW_EINVAL;  // one item per curve here; the value is not used
  (void)cudaGetLastError();

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FPW_ECUDA;
  DeviceSetup* ds = nullptr;
  int rc = setup_device(dev, &ds);
  if (rc != FPW_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // Every offset is checked before a kernel indexes the observations with it:
  // the host copy when given, else the device offsets read back through a
  // fixed buffer on the stack (no allocation).
  int64_t nobs = 0, prev = -1;
  if (offsets_host) {
    if (!offsets_chunk_ok(offsets_host, ncurves + 1, prev)) return FPW_EINVAL;
  } else {
    constexpr int64_t kChunk = 2048;
    int64_t buf[kChunk];
    for (int64_t q = 0; q <= ncurves; q += kChunk) {
      const int64_t cnt = (ncurves + 1 - q) < kChunk ? (ncurves + 1 - q) : kChunk;
      if (cudaMemcpyAsync(buf, offsets + q, sizeof(int64_t) * (size_t)cnt, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return FPW_ECUDA;
      if (!offsets_chunk_ok(buf, cnt, prev)) return FPW_EINVAL;
    }
  }
  nobs = prev;
  if (nobs > 0 && (!t || !x || !sigma)) return FPW_EINVAL;

  // kernel shape: as the tuned default, with the chunk sized to fit two blocks per SM
  const bool wide = p.accum != FPW_ACCUM_FP32;  // 16-byte bins
  TileShape sh{};
  sh.threads = p.threads ? p.threads : 128;
  sh.R = p.freqs_per_thread ? p.freqs_per_thread : (wide ? 2 : (M <= 24 ? 4 : 2));
  if (!tile_has_R(sh.R, p.accum, false)) return FPW_ENOTSUP;
  int NC = p.obs_chunk;
  if (!NC) {
    for (int blocks : {2, 1}) {
      for (int nc = 4096; nc >= 32; nc -= 32) {
        const size_t s = tile_smem_bytes(sh.threads, sh.R, M, nc, k, p.accum);
        if (s <= (size_t)ds->smem_optin && (s + 1024) * blocks <= (size_t)ds->smem_per_sm) {
          NC = nc;
          break;
        }
      }
      if (NC >= 256) break;
      NC = 0;
    }
    if (!NC) return FPW_ENOTSUP;
  }
  sh.obs_chunk = NC;
  sh.smem = tile_smem_bytes(sh.threads, sh.R, M, NC, k, p.accum);
  if (sh.smem > (size_t)ds->smem_optin) return FPW_ENOTSUP;
  const int bps = tile_max_blocks_per_sm(sh.R, p.phase_mode, p.accum, sh.threads, sh.smem);
  if (bps < 1) return FPW_ENOTSUP;

  // scratch layout (256-byte aligned sections); reject inputs that do not fit
  const size_t o_words = 0;  // counter, status (64 B), then the size-class histogram
  const size_t o_hist = o_words + 64;
  const size_t o_items = up256(o_hist + kSizeClasses * sizeof(unsigned));
  const size_t o_base = up256(o_items + (size_t)ncurves * sizeof(WorkItem));
  const size_t o_bad = up256(o_base + (size_t)(ncurves + 1) * sizeof(int32_t));
  const size_t o_cS = up256(o_bad + (size_t)ncurves);
  const size_t o_cI = up256(o_cS + (size_t)ncurves * k * sizeof(double));
  const size_t o_aw = up256(o_cI + (size_t)ncurves * k * sizeof(int32_t));
  const size_t end = o_aw + (size_t)(nobs + 2) * accum_bin_bytes(p.accum);
  if (end > kScratchBytes) return FPW_EINVAL;
  unsigned char* S = ds->scratch;
  unsigned* words = reinterpret_cast<unsigned*>(S + o_words);
  unsigned* hist = reinterpret_cast<unsigned*>(S + o_hist);
  WorkItem* items = reinterpret_cast<WorkItem*>(S + o_items);
  int32_t* cand_base = reinterpret_cast<int32_t*>(S + o_base);
  uint8_t* curve_bad = S + o_bad;
  double* cand_S = reinterpret_cast<double*>(S + o_cS);
  int32_t* cand_idx = reinterpret_cast<int32_t*>(S + o_cI);
  void* aw = S + o_aw;

  // counter, call status, histogram and per-curve flags must start at zero:
  // the array keeps whatever the previous call left in it
  if (cudaMemsetAsync(words, 0, o_items - o_words, st) != cudaSuccess) return FPW_ECUDA;
  if (cudaMemsetAsync(curve_bad, 0, (size_t)ncurves, st) != cudaSuccess) return FPW_ECUDA;
  {
    int64_t blocks = (ncurves + 1 + 255) / 256;
    blocks = blocks > 4096 ? 4096 : blocks;
    noalloc_count_kernel<<<(unsigned)blocks, 256, 0, st>>>(offsets, ncurves, hist, cand_base);
    noalloc_scan_kernel<<<1, 1, 0, st>>>(hist);
    noalloc_items_kernel<<<(unsigned)blocks, 256, 0, st>>>(offsets, ncurves, nfreq, hist, items);
    if (cudaGetLastError() != cudaSuccess) return FPW_ECUDA;
  }
  PrepArgs pa{};
  pa.t = t;
  pa.x = x;
  pa.sigma = sigma;
  pa.offsets = offsets;
  pa.ncurves = ncurves;
  pa.nobs = nobs;
  pa.freqs = freqs;
  pa.nfreq = nfreq;
  pa.aw = aw;
  pa.accum = p.accum;
  pa.curve_bad = curve_bad;
  pa.status = words + 1;
  if (launch_prep(pa, st) != cudaSuccess) return FPW_ECUDA;
  TileArgs ta{};
  ta.t = t;
  ta.offsets = offsets;
  ta.n_single = 0;
  ta.aw = aw;
  ta.freqs = freqs;
  ta.nfreq = nfreq;
  ta.items = items;
  ta.nitems = (int)ncurves;
  ta.counter = words;
  ta.status = words + 1;
  ta.curve_bad = curve_bad;
  ta.cand_S = k > 0 ? cand_S : nullptr;
  ta.cand_idx = k > 0 ? cand_idx : nullptr;
  ta.S_out = nullptr;
  ta.M = M;
  ta.k = k;
  ta.peak_raw = p.peak_mode == FPW_PEAK_RAW ? 1 : 0;
  ta.K = p.K;
  ta.obs_chunk = sh.obs_chunk;
  ta.inv_alpha2 = p.inv_alpha2;
  int grid = bps * ds->nsm;
  grid = grid < (int)ncurves ? grid : (int)ncurves;
  if (launch_tile(ta, sh, p.phase_mode, p.accum, grid, st) != cudaSuccess) return FPW_ECUDA;
  if (k > 0) {
    MergeArgs ma{};
    ma.cand_S = cand_S;
    ma.cand_idx = cand_idx;
    ma.cand_base = cand_base;
    ma.curve_bad = curve_bad;
    ma.status = words + 1;
    ma.ncurves = ncurves;
    ma.k = k;
    ma.topk_idx = topk_idx;
    ma.topk_S = topk_S;
    if (launch_merge(ma, st) != cudaSuccess) return FPW_ECUDA;
  }
  unsigned w = 0;
  if (cudaMemcpyAsync(&w, words + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FPW_ECUDA;
  if (w & kStatusTimeout) return FPW_ETIMEOUT;
  if (w & (kStatusData | kStatusGrid)) return FPW_EDATA;
  return FPW_OK;
}
