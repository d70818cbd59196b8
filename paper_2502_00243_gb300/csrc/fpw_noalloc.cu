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

__global__ void noalloc_items_kernel(WorkItem* items, int32_t* cand_base, int64_t C, int64_t F) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= C; c += (int64_t)gridDim.x * blockDim.x) {
    cand_base[c] = (int32_t)c;
    if (c < C) {
      WorkItem w;
      w.curve = (int32_t)c;
      w.f_lo = 0;
      w.f_hi = (int32_t)F;
      w.slot = (int32_t)c;
      items[c] = w;
    }
  }
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
  if (p.accum != FPW_ACCUM_FP32 && p.accum != FPW_ACCUM_FP64) return FPW_EINVAL;
  if (p.threads != 0 && (p.threads < 32 || p.threads > 512 || p.threads % 32 != 0)) return FPW_EINVAL;
  if (p.freqs_per_thread != 0 && !tile_supported_R(p.freqs_per_thread)) return FPW_EINVAL;
  if (p.obs_chunk != 0 && p.obs_chunk < 32) return FPW_EINVAL;
  (void)cudaGetLastError();

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FPW_ECUDA;
  DeviceSetup* ds = nullptr;
  int rc = setup_device(dev, &ds);
  if (rc != FPW_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // number of observations: from the host copy, else 8 bytes read back
  int64_t nobs = 0;
  if (offsets_host) {
    if (offsets_host[0] != 0) return FPW_EINVAL;
    for (int64_t c = 0; c < ncurves; ++c)
      if (offsets_host[c + 1] < offsets_host[c]) return FPW_EINVAL;
    nobs = offsets_host[ncurves];
  } else {
    if (cudaMemcpyAsync(&nobs, offsets + ncurves, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return FPW_ECUDA;
    if (nobs < 0) return FPW_EINVAL;
  }
  if (nobs > 0 && (!t || !x || !sigma)) return FPW_EINVAL;

  // kernel shape: as the tuned default, with the chunk sized to fit two blocks per SM
  const bool acc64 = p.accum == FPW_ACCUM_FP64;
  TileShape sh{};
  sh.threads = p.threads ? p.threads : 128;
  sh.R = p.freqs_per_thread ? p.freqs_per_thread : (acc64 ? 2 : (M <= 24 ? 4 : 2));
  int NC = p.obs_chunk;
  if (!NC) {
    for (int blocks : {2, 1}) {
      for (int nc = 4096; nc >= 32; nc -= 32) {
        const size_t s = tile_smem_bytes(sh.threads, sh.R, M, nc, k, acc64);
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
  sh.smem = tile_smem_bytes(sh.threads, sh.R, M, NC, k, acc64);
  if (sh.smem > (size_t)ds->smem_optin) return FPW_ENOTSUP;
  const int bps = tile_max_blocks_per_sm(sh.R, p.phase_mode, acc64, sh.threads, sh.smem);
  if (bps < 1) return FPW_ENOTSUP;

  // scratch layout (256-byte aligned sections); reject inputs that do not fit
  const size_t o_words = 0;
  const size_t o_items = up256(o_words + 64);
  const size_t o_base = up256(o_items + (size_t)ncurves * sizeof(WorkItem));
  const size_t o_bad = up256(o_base + (size_t)(ncurves + 1) * sizeof(int32_t));
  const size_t o_cS = up256(o_bad + (size_t)ncurves);
  const size_t o_cI = up256(o_cS + (size_t)ncurves * k * sizeof(double));
  const size_t o_aw = up256(o_cI + (size_t)ncurves * k * sizeof(int32_t));
  const size_t end = o_aw + (size_t)(nobs + 2) * (acc64 ? 16 : 8);
  if (end > kScratchBytes) return FPW_EINVAL;
  unsigned char* S = ds->scratch;
  unsigned* words = reinterpret_cast<unsigned*>(S + o_words);
  WorkItem* items = reinterpret_cast<WorkItem*>(S + o_items);
  int32_t* cand_base = reinterpret_cast<int32_t*>(S + o_base);
  uint8_t* curve_bad = S + o_bad;
  double* cand_S = reinterpret_cast<double*>(S + o_cS);
  int32_t* cand_idx = reinterpret_cast<int32_t*>(S + o_cI);
  void* aw = S + o_aw;

  // counter, call status and per-curve flags must start at zero: the array
  // keeps whatever the previous call left in it
  if (cudaMemsetAsync(words, 0, 64, st) != cudaSuccess) return FPW_ECUDA;
  if (cudaMemsetAsync(curve_bad, 0, (size_t)ncurves, st) != cudaSuccess) return FPW_ECUDA;
  {
    int64_t blocks = (ncurves + 1 + 255) / 256;
    blocks = blocks > 4096 ? 4096 : blocks;
    noalloc_items_kernel<<<(unsigned)blocks, 256, 0, st>>>(items, cand_base, ncurves, nfreq);
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
  pa.accum64 = acc64 ? 1 : 0;
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
  if (launch_tile(ta, sh, p.phase_mode, acc64, grid, st) != cudaSuccess) return FPW_ECUDA;
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
