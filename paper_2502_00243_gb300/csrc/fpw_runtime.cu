// Host runtime of the GB300 FPW library: the C ABI of include/fpw.h.
//
// Responsibilities: argument validation, the per-context device scratch
// (grow-only buffers), the batch planner (work items over curves and frequency
// segments, cost-sorted for the persistent kernel), kernel-shape selection,
// CUDA-graph capture and replay of repeated identical calls, the binary64
// plain form (one launch per curve), and the host-buffer end-to-end entry.
#include <algorithm>
#include <cmath>
#include <utility>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fpw_shared.cuh"

using namespace fpw;

namespace {

thread_local char g_last_cuda_error[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", what, cudaGetErrorString(e));
  if (getenv("FPW_DEBUG")) fprintf(stderr, "[fpw] %s\n", g_last_cuda_error);
  return e == cudaErrorMemoryAllocation ? FPW_ENOMEM : FPW_ECUDA;
}

#define FPW_CK(call)                                   \
  do {                                                 \
    cudaError_t fpw_e_ = (call);                       \
    if (fpw_e_ != cudaSuccess) return cuda_fail(fpw_e_, #call); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (bytes <= b.cap && b.p) return cudaSuccess;
  if (b.p) {
    cudaError_t e = cudaFree(b.p);  // synchronizes the device
    b.p = nullptr;
    b.cap = 0;
    if (e != cudaSuccess) return e;
  }
  size_t want = bytes < 256 ? 256 : bytes;
  want = (want + 255) & ~(size_t)255;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return e;
  }
  b.cap = want;
  return cudaSuccess;
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

template <typename T>
uint64_t mix(uint64_t h, const T& v) {
  return fnv1a(&v, sizeof(T), h);
}

struct Plan {
  uint64_t key = 0;
  TileShape shape{};
  int grid = 0;
  int nitems = 0;
  int nslots = 0;
  int max_rows = 0;  // most candidate rows (work items) of one curve
  DevBuf items, cand_base;
  void* host_stage = nullptr;  // pinned copy of items + cand_base, the source of the asynchronous upload
  uint64_t use = 0;
};

// A tuned kernel shape for bin counts in [M_lo, M_hi] and a typical curve size
// (observation-weighted mean N) in [n_lo, n_hi).
struct ShapeEntry {
  int M_lo, M_hi;
  int64_t n_lo, n_hi;
  int T, R, NC, items;
};

struct GraphEntry {
  uint64_t key = 0;
  cudaGraphExec_t exec = nullptr;
  uint64_t use = 0;
};

constexpr int kMaxPlans = 16;
constexpr int kMaxGraphs = 16;

}  // namespace

struct fpw_ctx {
  int device = 0;
  int nsm = 0;
  int smem_optin = 0;
  int smem_per_sm = 0;
  std::mutex mu;
  cudaStream_t last_stream = nullptr;
  cudaStream_t own_stream = nullptr;
  DevBuf aw, cand_S, cand_idx, curve_bad, words, dense, tile_dev;
  DevBuf sh_image, sh_scale, sh_S32, sh_step, sh_sink;  // shared-timestamp path scratch
  DevBuf dr_payload, dr_H0, dr_g, dr_tabs;                     // baseline-drift path scratch
  DevBuf h_off, h_t, h_x, h_sigma, h_freqs, h_idx, h_S;  // device copies for the host entry point
  std::vector<int64_t> off_host;                          // host copy of offsets (when not supplied)
  std::vector<Plan*> plans;
  std::vector<GraphEntry> graphs;
  std::vector<ShapeEntry> shapes;  // tuned shapes (latest entry wins)
  uint64_t tick = 0;
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // pairs (start, stop) of recorded tile launches
  size_t ev_used = 0;           // events in use (even count)
  TileShape last_shape{};       // shape and grid of the latest tile-kernel call
  int last_grid = 0;
  long long wait_clocks = 0;    // shared-timestamp pipeline wait limit (0: default)
};

namespace {

void free_buf(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

// Frees a plan; cudaFree synchronizes the device first, so its upload has ended.
void free_plan(Plan* p) {
  free_buf(p->items);
  free_buf(p->cand_base);
  if (p->host_stage) cudaFreeHost(p->host_stage);
  delete p;
}

// Discard a stale error left by an earlier, unrelated runtime call so that the
// launch checks below report only this call's errors.
void clear_stale_error() { (void)cudaGetLastError(); }

int status_to_code(unsigned s) {
  if (s & kStatusTimeout) return FPW_ETIMEOUT;
  if (s & (kStatusData | kStatusGrid)) return FPW_EDATA;
  return FPW_OK;
}

bool valid_params(const fpw_params& p) {
  if (!(p.inv_alpha2 >= 0.0) || !std::isfinite(p.inv_alpha2)) return false;
  if (p.phase_mode != FPW_PHASE_FIXED64 && p.phase_mode != FPW_PHASE_FP64 && p.phase_mode != FPW_PHASE_FP32)
    return false;
  if (p.accum != FPW_ACCUM_FP32 && p.accum != FPW_ACCUM_FP64 && p.accum != FPW_ACCUM_FP32_COMP) return false;
  if (p.K < 1) return false;
  if (p.peak_mode != FPW_PEAK_LOCALMAX && p.peak_mode != FPW_PEAK_RAW) return false;
  if (p.threads != 0 && (p.threads < 32 || p.threads > 512 || p.threads % 32 != 0)) return false;
  if (p.freqs_per_thread != 0 && !tile_supported_R(p.freqs_per_thread)) return false;
  if (p.obs_chunk != 0 && p.obs_chunk < 32) return false;
  if (p.items_per_slot < 0) return false;
  return true;
}

// Kernel shape: T threads, R frequencies per thread, NC observations per pass.
// Per-thread bins take R*M*T*(8|16) bytes (16 for binary64 and compensated
// sums); the observation chunk takes NC*(16 + 8|16) bytes. Precedence: explicit params > the context's tuned
// table (fpw_ctx_set_shape) > the built-in defaults, which were measured on a
// GB300 with ZTF-like curves (threads x frequencies-per-thread sweeps at
// M = 10, 16, 20, 24, 30, 40, 50): R = 8 for M <= 12, R = 6 for M <= 16, R = 5
// for M <= 20, R = 4 for M <= 25, R = 3 for M <= 33 (R = 2 for these when the
// typical curve has fewer than 300 observations, as measured at M = 20; R = 6, 5
// and 3 for FP32 sums of one M only, else 4 and 2), R = 2 up to M = 64, R = 1
// beyond, T = 128 (halved while the bins alone do not fit): up to about 100 bin
// pairs per thread keep two blocks of four warps per SM and spread each
// observation's broadcast over the most frequencies. NC: the largest chunk that
// keeps two resident blocks per SM (one stages while the other accumulates) if
// that is at least 128 observations, else one block per SM.
int choose_shape(fpw_ctx* ctx, const fpw_params& p, int M, int k, int64_t max_n, int64_t n_typ, int ngroups,
                 TileShape& out) {
  const bool wide = p.accum != FPW_ACCUM_FP32;  // 16-byte bins
  int T = 128, R = 4, NC = 0, items = 8;
  if (wide)
    R = 2;
  else if (M <= 12)
    R = 8;
  else if (M <= 16 && ngroups == 0)
    R = n_typ < 300 ? 2 : 6;
  else if (M <= 20 && ngroups == 0)
    R = n_typ < 300 ? 2 : 5;
  else if (M <= 24 || (M <= 25 && ngroups == 0))
    R = n_typ < 300 ? 2 : 4;
  else if (M <= 33 && ngroups == 0)
    R = n_typ < 300 ? 2 : 3;
  else if (M <= 40 || (M <= 50 && ngroups == 0))  // several M at M_max = 40: 1.23e12 against 1.17e12 at T = 256, R = 1
    R = 2;
  else if (M <= 50) {  // several M: the per-frequency combination favours more warps
    T = 256;
    R = 1;
  } else if (M <= 64) {  // two blocks of 6 warps per SM (T = 128, R = 2 leaves one block of 4)
    T = 192;
    R = 1;
    if (ngroups > 0) {  // several M at M_max = 60: three blocks of 4 warps, 256 observations per pass
      T = 128;          // (1.010e12 evaluations/s against 0.992e12 for two blocks of 6 warps)
      NC = 256;
    }
  } else
    R = 1;
  for (const ShapeEntry& e : ctx->shapes)
    if (M >= e.M_lo && M <= e.M_hi && n_typ >= e.n_lo && n_typ < e.n_hi) {
      T = e.T;
      R = e.R;
      NC = e.NC;
      items = e.items ? e.items : 8;
    }
  if (ngroups > 0 && T > 256) T = 256;  // the several-M kernel's launch bound (table entries may be wider)
  // R = 3 and 6 exist for FP32 sums of one M only: a table entry tuned there
  // gives the neighbouring instantiated R to the other kernels
  if (!tile_has_R(R, p.accum, ngroups > 0)) R = (R == 3) ? 2 : 4;
  if (p.threads) T = p.threads;
  if (p.items_per_slot) items = p.items_per_slot;
  if (p.freqs_per_thread) R = p.freqs_per_thread;
  if (!tile_has_R(R, p.accum, ngroups > 0)) return FPW_ENOTSUP;
  if (p.obs_chunk) NC = p.obs_chunk;
  const bool fixedT = p.threads != 0;
  while (!fixedT && T > 32 && tile_smem_bytes(T, R, M, 32, k, p.accum, ngroups) > (size_t)ctx->smem_optin) T /= 2;
  const int64_t want_nc = std::max<int64_t>(32, ((max_n + 31) / 32) * 32);
  const size_t per_sm = (size_t)ctx->smem_per_sm;
  auto fits = [&](int blocks, int nc) {
    const size_t s = tile_smem_bytes(T, R, M, nc, k, p.accum, ngroups);
    return s <= (size_t)ctx->smem_optin && (s + 1024) * blocks <= per_sm;
  };
  if (!NC) {
    for (int blocks : {2, 1}) {
      int lo = 32, hi = (int)std::min<int64_t>(want_nc, 1 << 16);
      if (!fits(blocks, lo)) continue;
      while (lo < hi) {  // largest multiple of 32 that fits
        int mid = ((lo + hi + 32) / 64) * 32;
        if (mid <= lo) mid = lo + 32;
        if (mid > hi) mid = hi;
        if (fits(blocks, mid))
          lo = mid;
        else
          hi = mid - 32;
      }
      // too small a chunk: one block per SM instead (two blocks with 128-160
      // observations per pass ran M = 20, R = 5 at 2.0e12 evals/s, one block
      // with a larger chunk 1.5e12)
      if (blocks == 2 && lo < 128 && lo < want_nc) continue;
      NC = lo;
      break;
    }
    if (!NC) return FPW_ENOTSUP;  // the bins alone exceed shared memory
  }
  const size_t smem = tile_smem_bytes(T, R, M, NC, k, p.accum, ngroups);
  if (smem > (size_t)ctx->smem_optin) return FPW_ENOTSUP;
  out.threads = T;
  out.R = R;
  out.obs_chunk = NC;
  out.smem = smem;
  out.items = items;
  return FPW_OK;
}

// Work items: each curve's frequency range split into segments of whole tiles
// so that every resident block gets about sh.items items (load balance), sorted by
// cost (observations x frequencies) descending; candidate rows per curve in
// curve order. The tables are uploaded from a pinned copy, ordered on `st`.
Plan* build_plan(fpw_ctx* ctx, const int64_t* off, int64_t C, int64_t F, const TileShape& sh, int blocks_per_sm,
                 uint64_t key, cudaStream_t st, int* err) {
  *err = FPW_OK;
  const int64_t Wown = (int64_t)sh.threads * sh.R - 2;
  const int64_t tiles = (F + Wown - 1) / Wown;
  const int resident = std::max(1, blocks_per_sm * ctx->nsm);
  double total = 0.0;
  for (int64_t c = 0; c < C; ++c) total += (double)(off[c + 1] - off[c] + 32) * (double)F;
  const double target = std::max(total / ((double)sh.items * resident), 32.0 * (double)Wown * 16.0);
  std::vector<double> ccv((size_t)C);
  std::vector<int64_t> nseg((size_t)C);
  bool all_split = C > 1;
  for (int64_t c = 0; c < C; ++c) {
    const double cc = (double)(off[c + 1] - off[c] + 32) * (double)F;
    ccv[(size_t)c] = cc;
    int64_t n = (int64_t)std::llround(cc / target);
    // A curve that would be cut finer than three tiles per item (a single long
    // curve, cut for load balance) gets whole rounds of the resident blocks,
    // each item at least three tiles: an item's prologue, restaging and
    // candidate row cost about a tile's latency, and equal items that do not
    // fill whole rounds leave blocks idle. 1000 observations x 1e6
    // frequencies: 0.635 -> 0.60 ms of tile kernel, 0.76 -> 0.67 ms per call.
    const int64_t rounds = tiles / (3 * (int64_t)resident);
    if (n > tiles / 3 && rounds >= 1) n = rounds * resident;
    n = std::max<int64_t>(1, std::min<int64_t>(n, tiles));
    nseg[(size_t)c] = n;
    if (n < 2) all_split = false;
  }
  // Every curve cut (a few long curves): the item count is made whole rounds
  // of the resident blocks, shared by cost with the largest remainders (20
  // equal curves over 2e6 frequencies and 152 blocks: 1220 items, a ninth
  // round nearly empty, became 1216).
  int64_t nall = 0;
  for (int64_t c = 0; c < C; ++c) nall += nseg[(size_t)c];
  if (all_split && nall >= resident && nall % resident != 0) {  // fewer items: the minimum item size binds
    const int64_t want = std::max<int64_t>(resident, (nall + resident / 2) / resident * resident);
    std::vector<std::pair<double, int64_t>> frac;
    int64_t got = 0;
    for (int64_t c = 0; c < C; ++c) {
      const double share = (double)want * ccv[(size_t)c] / total;
      const int64_t f = std::max<int64_t>(1, std::min<int64_t>((int64_t)std::floor(share), tiles));
      nseg[(size_t)c] = f;
      got += f;
      if (f < tiles) frac.emplace_back(share - std::floor(share), c);
    }
    std::stable_sort(frac.begin(), frac.end(), [](const std::pair<double, int64_t>& x, const std::pair<double, int64_t>& y) {
      return x.first > y.first;
    });
    for (size_t i = 0; i < frac.size() && got < want; ++i, ++got) nseg[(size_t)frac[i].second] += 1;
  }
  std::vector<WorkItem> items;
  std::vector<double> cost;
  std::vector<int32_t> base((size_t)C + 1, 0);
  items.reserve((size_t)C);
  for (int64_t c = 0; c < C; ++c) {
    const double cc = ccv[(size_t)c];
    const int64_t ns = nseg[(size_t)c];
    base[c + 1] = base[c] + (int32_t)ns;
    for (int64_t q = 0; q < ns; ++q) {
      const int64_t t0 = tiles * q / ns, t1 = tiles * (q + 1) / ns;
      WorkItem w;
      w.curve = (int32_t)c;
      w.f_lo = (int32_t)(t0 * Wown);
      w.f_hi = (int32_t)std::min<int64_t>(F, t1 * Wown);
      w.slot = base[c] + (int32_t)q;
      items.push_back(w);
      cost.push_back(cc * (double)(t1 - t0) / (double)tiles);
    }
  }
  std::vector<int> order(items.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<WorkItem> sorted(items.size());
  for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];

  Plan* pl = new (std::nothrow) Plan();
  if (!pl) {
    *err = FPW_ENOMEM;
    return nullptr;
  }
  pl->key = key;
  pl->shape = sh;
  pl->nitems = (int)sorted.size();
  pl->nslots = base[C];
  for (int64_t c = 0; c < C; ++c) pl->max_rows = std::max(pl->max_rows, base[c + 1] - base[c]);
  pl->grid = std::max(1, std::min(resident, pl->nitems));
  const size_t ib = sorted.size() * sizeof(WorkItem), bb = base.size() * sizeof(int32_t);
  cudaError_t e = ensure(pl->items, ib);
  if (e == cudaSuccess) e = ensure(pl->cand_base, bb);
  if (e == cudaSuccess) e = cudaMallocHost(&pl->host_stage, ib + bb);
  if (e == cudaSuccess) {
    memcpy(pl->host_stage, sorted.data(), ib);
    memcpy(static_cast<char*>(pl->host_stage) + ib, base.data(), bb);
    e = cudaMemcpyAsync(pl->items.p, pl->host_stage, ib, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pl->cand_base.p, static_cast<char*>(pl->host_stage) + ib, bb, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    *err = cuda_fail(e, "plan upload");
    free_plan(pl);
    return nullptr;
  }
  return pl;
}

Plan* get_plan(fpw_ctx* ctx, const int64_t* off, int64_t C, int64_t F, const TileShape& sh, int blocks_per_sm,
               cudaStream_t st, int* err) {
  uint64_t key = fnv1a(off, sizeof(int64_t) * (size_t)(C + 1));
  key = mix(key, C);
  key = mix(key, F);
  key = mix(key, sh.threads);
  key = mix(key, sh.R);
  key = mix(key, sh.obs_chunk);
  key = mix(key, sh.smem);
  key = mix(key, sh.items);
  key = mix(key, blocks_per_sm);
  for (Plan* p : ctx->plans)
    if (p->key == key) {
      p->use = ++ctx->tick;
      *err = FPW_OK;
      return p;
    }
  Plan* p = build_plan(ctx, off, C, F, sh, blocks_per_sm, key, st, err);
  if (!p) return nullptr;
  p->use = ++ctx->tick;
  if ((int)ctx->plans.size() >= kMaxPlans) {
    auto it = std::min_element(ctx->plans.begin(), ctx->plans.end(),
                               [](const Plan* a, const Plan* b) { return a->use < b->use; });
    // graphs may reference the evicted plan's buffers: drop them all
    for (GraphEntry& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
    free_plan(*it);
    ctx->plans.erase(it);
  }
  ctx->plans.push_back(p);
  return p;
}

int check_offsets(const int64_t* off, int64_t C) {
  if (off[0] != 0) return FPW_EINVAL;
  for (int64_t c = 0; c < C; ++c)
    if (off[c + 1] < off[c]) return FPW_EINVAL;
  if (off[C] > ((int64_t)1 << 40)) return FPW_EINVAL;
  return FPW_OK;
}

struct BatchCall {
  cudaStream_t stream;
  fpw_params p;
  const int64_t* offsets;  // device, or NULL for one curve
  const int64_t* off_h;    // host offsets [C+1]
  int64_t C;
  const double *t, *x, *sigma, *freqs;
  int64_t F;
  int M, k;
  int32_t* topk_idx;
  float* topk_S;
  double* S_out;
  int ngroups;              // several-M call: groups g (M = M_max / g); 0 = single M
  int groups[kMaxGroups];
  int32_t* topk_off;        // several-M call: offset of each reported peak
  int32_t* bins_out;        // bin dump of frequencies [bins_k0, bins_k1), or NULL
  int64_t bins_k0, bins_k1;
};

void drop_graphs(fpw_ctx* ctx) {
  for (GraphEntry& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
}

// Enqueue prep -> persistent tile kernel -> merge -> status latch.
int enqueue_tile_path(fpw_ctx* ctx, const BatchCall& b, Plan* pl, unsigned* words, cudaStream_t st) {
  const int64_t nobs = b.off_h[b.C];
  FPW_CK(cudaMemsetAsync(words, 0, 2 * sizeof(unsigned), st));
  FPW_CK(cudaMemsetAsync(ctx->curve_bad.p, 0, (size_t)b.C, st));
  PrepArgs pa{};
  pa.t = b.t;
  pa.x = b.x;
  pa.sigma = b.sigma;
  pa.offsets = b.offsets;
  pa.ncurves = b.C;
  pa.nobs = nobs;
  pa.freqs = b.freqs;
  pa.nfreq = b.F;
  pa.aw = ctx->aw.p;
  pa.accum = b.p.accum;
  pa.curve_bad = static_cast<uint8_t*>(ctx->curve_bad.p);
  pa.status = words + 1;
  FPW_CK(launch_prep(pa, st));
  const int W = pl->shape.threads * pl->shape.R;
  const int64_t tiles = (b.F + (W - 2) - 1) / (W - 2);
  FPW_CK(launch_tile_dev(b.freqs, b.F, W, tiles, static_cast<double*>(ctx->tile_dev.p), st));
  TileArgs ta{};
  ta.t = b.t;
  ta.offsets = b.offsets;
  ta.n_single = b.offsets ? 0 : nobs;
  ta.aw = ctx->aw.p;
  ta.freqs = b.freqs;
  ta.nfreq = b.F;
  ta.items = static_cast<const WorkItem*>(pl->items.p);
  ta.nitems = pl->nitems;
  ta.counter = words;
  ta.status = words + 1;
  ta.curve_bad = static_cast<const uint8_t*>(ctx->curve_bad.p);
  ta.cand_S = b.k > 0 ? static_cast<double*>(ctx->cand_S.p) : nullptr;
  ta.cand_idx = b.k > 0 ? static_cast<int32_t*>(ctx->cand_idx.p) : nullptr;
  ta.S_out = b.S_out;
  ta.M = b.M;
  ta.k = b.k;
  ta.peak_raw = b.p.peak_mode == FPW_PEAK_RAW ? 1 : 0;
  ta.K = b.p.K;
  ta.obs_chunk = pl->shape.obs_chunk;
  ta.inv_alpha2 = b.p.inv_alpha2;
  ta.tile_dev = static_cast<const double*>(ctx->tile_dev.p);
  ta.ngroups = b.ngroups;
  for (int q = 0; q < b.ngroups; ++q) ta.group_g[q] = b.groups[q];
  ta.group_rows = pl->nslots;
  ta.bins_out = b.bins_out;
  ta.bins_k0 = b.bins_k0;
  ta.bins_k1 = b.bins_k1;
  ta.bins_nobs = nobs;
  const bool timed = ctx->timing && !b.p.use_graph;
  if (timed) {
    while (ctx->ev.size() < ctx->ev_used + 2) {
      cudaEvent_t e;
      FPW_CK(cudaEventCreate(&e));
      ctx->ev.push_back(e);
    }
    FPW_CK(cudaEventRecord(ctx->ev[ctx->ev_used], st));
  }
  FPW_CK(launch_tile(ta, pl->shape, b.p.phase_mode, b.p.accum, pl->grid, st));
  if (timed) {
    FPW_CK(cudaEventRecord(ctx->ev[ctx->ev_used + 1], st));
    ctx->ev_used += 2;
  }
  if (b.k > 0) {
    const int ng = b.ngroups > 0 ? b.ngroups : 1;
    for (int q = 0; q < ng; ++q) {
      const int64_t rows = (int64_t)q * pl->nslots * b.k;
      MergeArgs ma{};
      ma.cand_S = static_cast<const double*>(ctx->cand_S.p) + rows;
      ma.cand_idx = static_cast<const int32_t*>(ctx->cand_idx.p) + rows;
      ma.cand_base = static_cast<const int32_t*>(pl->cand_base.p);
      ma.curve_bad = static_cast<const uint8_t*>(ctx->curve_bad.p);
      ma.status = words + 1;
      ma.ncurves = b.C;
      ma.k = b.k;
      ma.topk_idx = b.topk_idx + (int64_t)q * b.k;
      ma.topk_S = b.topk_S + (int64_t)q * b.k;
      ma.out_stride = ng * b.k;
      ma.topk_off = b.ngroups > 0 ? b.topk_off + (int64_t)q * b.k : nullptr;
      ma.max_rows = pl->max_rows;
      FPW_CK(launch_merge(ma, st));
    }
  }
  FPW_CK(launch_latch(words, st));
  return FPW_OK;
}

int run_tile_path(fpw_ctx* ctx, const BatchCall& b) {
  int64_t max_n = 0;
  double sn = 0.0, sn2 = 0.0;
  for (int64_t c = 0; c < b.C; ++c) {
    const int64_t n = b.off_h[c + 1] - b.off_h[c];
    max_n = std::max(max_n, n);
    sn += (double)n;
    sn2 += (double)n * (double)n;
  }
  const int64_t n_typ = sn > 0.0 ? (int64_t)(sn2 / sn) : 0;  // observation-weighted mean curve size
  TileShape sh{};
  int rc = choose_shape(ctx, b.p, b.M, b.k, max_n, n_typ, b.ngroups, sh);
  if (rc != FPW_OK) return rc;
  const int bps = tile_max_blocks_per_sm(sh.R, b.p.phase_mode, b.p.accum, sh.threads, sh.smem, b.ngroups > 0,
                                         b.bins_out != nullptr, multi_spec_of(b.M, b.ngroups, b.groups));
  if (bps < 1) return FPW_ENOTSUP;
  Plan* pl = get_plan(ctx, b.off_h, b.C, b.F, sh, bps, b.stream, &rc);
  if (!pl) return rc;
  ctx->last_shape = sh;
  ctx->last_grid = pl->grid;
  const int64_t nobs = b.off_h[b.C];
  // scratch (grow-only; growing invalidates captured graphs)
  void* before[6] = {ctx->aw.p, ctx->cand_S.p, ctx->cand_idx.p, ctx->curve_bad.p, ctx->words.p, ctx->tile_dev.p};
  cudaError_t e = ensure(ctx->aw, (size_t)(nobs + 2) * accum_bin_bytes(b.p.accum));
  {
    const int64_t Wown = (int64_t)sh.threads * sh.R - 2;
    if (e == cudaSuccess) e = ensure(ctx->tile_dev, sizeof(double) * (size_t)((b.F + Wown - 1) / Wown + 1));
  }
  const size_t ng = (size_t)(b.ngroups > 0 ? b.ngroups : 1);
  if (e == cudaSuccess && b.k > 0) e = ensure(ctx->cand_S, ng * pl->nslots * b.k * sizeof(double));
  if (e == cudaSuccess && b.k > 0) e = ensure(ctx->cand_idx, ng * pl->nslots * b.k * sizeof(int32_t));
  if (e == cudaSuccess) e = ensure(ctx->curve_bad, (size_t)b.C + 16);
  if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
  void* after[6] = {ctx->aw.p, ctx->cand_S.p, ctx->cand_idx.p, ctx->curve_bad.p, ctx->words.p, ctx->tile_dev.p};
  if (memcmp(before, after, sizeof(before)) != 0) drop_graphs(ctx);
  unsigned* words = static_cast<unsigned*>(ctx->words.p);

  if (!b.p.use_graph || b.bins_out) return enqueue_tile_path(ctx, b, pl, words, b.stream);

  uint64_t gk = mix(pl->key, (const void*)b.stream);
  for (const void* q : {(const void*)b.offsets, (const void*)b.t, (const void*)b.x, (const void*)b.sigma,
                        (const void*)b.freqs, (const void*)b.topk_idx, (const void*)b.topk_S, (const void*)b.S_out})
    gk = mix(gk, q);
  gk = mix(gk, b.C);
  gk = mix(gk, b.F);
  gk = mix(gk, b.M);
  gk = mix(gk, b.k);
  gk = mix(gk, b.p.inv_alpha2);
  gk = mix(gk, b.p.phase_mode);
  gk = mix(gk, b.p.accum);
  gk = mix(gk, b.p.K);
  gk = mix(gk, b.p.peak_mode);
  gk = mix(gk, b.ngroups);
  for (int q = 0; q < b.ngroups; ++q) gk = mix(gk, b.groups[q]);
  gk = mix(gk, (const void*)b.topk_off);
  gk = mix(gk, ctx->aw.p);
  gk = mix(gk, ctx->cand_S.p);
  gk = mix(gk, ctx->cand_idx.p);
  gk = mix(gk, ctx->curve_bad.p);
  gk = mix(gk, ctx->tile_dev.p);
  gk = mix(gk, pl);
  for (GraphEntry& g : ctx->graphs)
    if (g.key == gk) {
      g.use = ++ctx->tick;
      FPW_CK(cudaGraphLaunch(g.exec, b.stream));
      return FPW_OK;
    }
  // Capture on the context's own stream (the legacy default stream cannot be
  // captured); the instantiated graph is launched on the caller's stream.
  cudaGraph_t graph = nullptr;
  FPW_CK(cudaStreamBeginCapture(ctx->own_stream, cudaStreamCaptureModeThreadLocal));
  rc = enqueue_tile_path(ctx, b, pl, words, ctx->own_stream);
  cudaError_t ec = cudaStreamEndCapture(ctx->own_stream, &graph);
  if (rc != FPW_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  ec = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ec != cudaSuccess) return cuda_fail(ec, "cudaGraphInstantiate");
  if ((int)ctx->graphs.size() >= kMaxGraphs) {
    auto it = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                               [](const GraphEntry& a, const GraphEntry& b2) { return a.use < b2.use; });
    cudaGraphExecDestroy(it->exec);
    ctx->graphs.erase(it);
  }
  GraphEntry ge;
  ge.key = gk;
  ge.exec = exec;
  ge.use = ++ctx->tick;
  ctx->graphs.push_back(ge);
  FPW_CK(cudaGraphLaunch(exec, b.stream));
  return FPW_OK;
}

// The binary64 plain form: per curve one periodogram launch (and one top-k launch).
int run_plain_path(fpw_ctx* ctx, const BatchCall& b) {
  if (plain_smem_bytes(b.M) > (size_t)ctx->smem_optin) return FPW_ENOTSUP;  // binary64 bins of one block
  unsigned* words = static_cast<unsigned*>(ctx->words.p);
  FPW_CK(cudaMemsetAsync(words, 0, 2 * sizeof(unsigned), b.stream));
  // validate frequencies (and observations) once for the status word
  PrepArgs pa{};
  pa.t = b.t;
  pa.x = b.x;
  pa.sigma = b.sigma;
  pa.offsets = b.offsets;
  pa.ncurves = b.C;
  pa.nobs = b.off_h[b.C];
  pa.freqs = b.freqs;
  pa.nfreq = b.F;
  pa.aw = nullptr;
  FPW_CK(ensure(ctx->curve_bad, (size_t)b.C + 16));
  FPW_CK(cudaMemsetAsync(ctx->curve_bad.p, 0, (size_t)b.C, b.stream));
  pa.curve_bad = static_cast<uint8_t*>(ctx->curve_bad.p);
  pa.status = words + 1;
  FPW_CK(launch_prep(pa, b.stream));
  if (!b.S_out) FPW_CK(ensure(ctx->dense, (size_t)b.F * sizeof(double)));
  for (int64_t c = 0; c < b.C; ++c) {
    const int64_t o = b.off_h[c], n = b.off_h[c + 1] - o;
    double* S = b.S_out ? b.S_out + c * b.F : static_cast<double*>(ctx->dense.p);
    PlainArgs a{};
    a.t = b.t + o;
    a.x = b.x + o;
    a.sigma = b.sigma + o;
    a.n = n;
    a.freqs = b.freqs;
    a.nfreq = b.F;
    a.M = b.M;
    a.inv_alpha2 = b.p.inv_alpha2;
    a.S_out = S;
    a.status = words + 1;
    a.bins_out = b.bins_out;
    a.bins_k0 = b.bins_k0;
    a.bins_k1 = b.bins_k1;
    a.bins_nobs = b.off_h[b.C];
    a.bins_base = o;
    FPW_CK(launch_plain(a, b.stream));
    if (b.k > 0) {
      DenseTopkArgs d{};
      d.S = S;
      d.nfreq = b.F;
      d.k = b.k;
      d.peak_raw = b.p.peak_mode == FPW_PEAK_RAW ? 1 : 0;
      d.topk_idx = b.topk_idx + c * b.k;
      d.topk_S = b.topk_S + c * b.k;
      FPW_CK(launch_dense_topk(d, b.stream));
    }
  }
  FPW_CK(launch_latch(words, b.stream));
  return FPW_OK;
}

int batch_impl(fpw_ctx* ctx, BatchCall& b) {
  if (b.C == 0) return FPW_OK;
  if (b.F == 0) {
    if (b.k > 0) FPW_CK(launch_fill_topk(b.topk_idx, b.topk_S, b.C * b.k, b.stream));
    return FPW_OK;
  }
  if (b.F > ((int64_t)1 << 31) - 1024 || b.C > ((int64_t)1 << 31) - 1) return FPW_EINVAL;
  if (b.p.phase_mode == FPW_PHASE_FP64) return run_plain_path(ctx, b);
  return run_tile_path(ctx, b);
}

int sync_status(fpw_ctx* ctx, cudaStream_t st, int rc) {
  if (rc != FPW_OK) return rc;
  FPW_CK(cudaStreamSynchronize(st));
  unsigned w = 0;
  FPW_CK(cudaMemcpy(&w, static_cast<unsigned*>(ctx->words.p) + 1, sizeof(unsigned), cudaMemcpyDeviceToHost));
  return status_to_code(w);
}

std::mutex g_default_mu;
fpw_ctx* g_default[64] = {nullptr};

fpw_ctx* default_ctx(int* rc) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *rc = FPW_ECUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_default_mu);
  if (!g_default[dev]) {
    *rc = fpw_ctx_create(&g_default[dev], dev);
    if (*rc != FPW_OK) {
      g_default[dev] = nullptr;
      return nullptr;
    }
  }
  *rc = FPW_OK;
  return g_default[dev];
}

// Shared body of the batched entry points (arguments checked by the caller
// for the parts specific to each).
int batch_entry(fpw_ctx* ctx, void* stream, const fpw_params* params, const int64_t* offsets,
                const int64_t* offsets_host, int64_t ncurves, const double* t, const double* x, const double* sigma,
                const double* freqs, int64_t nfreq, int M, int k, int32_t* topk_idx, float* topk_S, double* S_out,
                int32_t* bins_out, int64_t k0, int64_t k1) {
  if (ncurves > 0 && !offsets) return FPW_EINVAL;
  if (ncurves > 0 && nfreq > 0 && !freqs) return FPW_EINVAL;
  fpw_params p;
  fpw_params_default(&p);
  if (params) p = *params;
  if (!valid_params(p)) return FPW_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return FPW_ECUDA;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_stale_error();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ctx->last_stream = st;
  if (ncurves == 0) return FPW_OK;
  const int64_t* off_h = offsets_host;
  if (!off_h) {
    ctx->off_host.resize((size_t)ncurves + 1);
    FPW_CK(cudaMemcpyAsync(ctx->off_host.data(), offsets, sizeof(int64_t) * (size_t)(ncurves + 1),
                           cudaMemcpyDeviceToHost, st));
    FPW_CK(cudaStreamSynchronize(st));
    off_h = ctx->off_host.data();
  }
  if (check_offsets(off_h, ncurves) != FPW_OK) return FPW_EINVAL;
  if (off_h[ncurves] > 0 && (!t || !x || !sigma)) return FPW_EINVAL;
  BatchCall b{};
  b.stream = st;
  b.p = p;
  b.offsets = offsets;
  b.off_h = off_h;
  b.C = ncurves;
  b.t = t;
  b.x = x;
  b.sigma = sigma;
  b.freqs = freqs;
  b.F = nfreq;
  b.M = M;
  b.k = k;
  b.topk_idx = topk_idx;
  b.topk_S = topk_S;
  b.S_out = S_out;
  b.bins_out = off_h[ncurves] > 0 ? bins_out : nullptr;
  b.bins_k0 = k0;
  b.bins_k1 = k1;
  return batch_impl(ctx, b);
}

}  // namespace

extern "C" {

void fpw_params_default(fpw_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->inv_alpha2 = 0.0;
  p->phase_mode = FPW_PHASE_FIXED64;
  p->accum = FPW_ACCUM_FP32;
  p->K = 256;
  p->peak_mode = FPW_PEAK_LOCALMAX;
  p->use_graph = 0;
}

int fpw_version(void) { return 2; }

const char* fpw_strerror(int s) {
  switch (s) {
    case FPW_OK: return "ok";
    case FPW_EINVAL: return "invalid argument";
    case FPW_EDATA: return "invalid data (sigma <= 0 or a non-finite input)";
    case FPW_ENOMEM: return "out of memory";
    case FPW_ECUDA: return "CUDA runtime error";
    case FPW_ETIMEOUT: return "bounded device wait timed out";
    case FPW_ENOTSUP: return "unsupported combination of options";
    default: return "unknown status";
  }
}

const char* fpw_last_cuda_error(void) { return g_last_cuda_error; }

int fpw_ctx_create(fpw_ctx** out, int device) {
  if (!out) return FPW_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FPW_EINVAL;
  DeviceGuard g(device);
  if (!g.ok) return FPW_ECUDA;
  fpw_ctx* ctx = new (std::nothrow) fpw_ctx();
  if (!ctx) return FPW_ENOMEM;
  ctx->device = device;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, device);
  if (e == cudaSuccess) {
    ctx->nsm = prop.multiProcessorCount;
    ctx->smem_optin = (int)prop.sharedMemPerBlockOptin;
    ctx->smem_per_sm = (int)prop.sharedMemPerMultiprocessor;
    e = tile_init_attributes(ctx->smem_optin);
  }
  if (e == cudaSuccess) e = plain_init_attributes(ctx->smem_optin);
  if (e == cudaSuccess && (size_t)ctx->smem_optin >= shared_smem_bytes()) e = shared_init_attributes();
  if (e == cudaSuccess) e = drift_init_attributes(ctx->smem_optin);
  if (e == cudaSuccess) e = ensure(ctx->words, 64);
  if (e == cudaSuccess) e = cudaMemset(ctx->words.p, 0, 64);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    int rc = cuda_fail(e, "fpw_ctx_create");
    free_buf(ctx->words);
    delete ctx;
    return rc;
  }
  *out = ctx;
  return FPW_OK;
}

int fpw_ctx_destroy(fpw_ctx* ctx) {
  if (!ctx) return FPW_OK;
  {
    DeviceGuard g(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaDeviceSynchronize();
    drop_graphs(ctx);
    for (Plan* p : ctx->plans) free_plan(p);
    ctx->plans.clear();
    for (DevBuf* b : {&ctx->aw, &ctx->cand_S, &ctx->cand_idx, &ctx->curve_bad, &ctx->words, &ctx->dense, &ctx->tile_dev, &ctx->h_off,
                      &ctx->h_t, &ctx->h_x, &ctx->h_sigma, &ctx->h_freqs, &ctx->h_idx, &ctx->h_S, &ctx->sh_image,
                      &ctx->sh_scale, &ctx->sh_S32, &ctx->sh_step, &ctx->sh_sink, &ctx->dr_payload,
                      &ctx->dr_H0, &ctx->dr_g, &ctx->dr_tabs})
      free_buf(*b);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  }
  delete ctx;
  return FPW_OK;
}

int fpw_ctx_set_shape(fpw_ctx* ctx, int M_lo, int M_hi, int64_t n_lo, int64_t n_hi, int threads, int freqs_per_thread,
                      int obs_chunk, int items_per_slot) {
  if (!ctx || M_lo < 1 || M_hi < M_lo || n_lo < 0 || n_hi <= n_lo) return FPW_EINVAL;
  if (threads < 32 || threads > 512 || threads % 32 != 0 || !tile_supported_R(freqs_per_thread)) return FPW_EINVAL;
  if ((obs_chunk != 0 && obs_chunk < 32) || items_per_slot < 0) return FPW_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ShapeEntry e{M_lo, M_hi, n_lo, n_hi, threads, freqs_per_thread, obs_chunk, items_per_slot};
  ctx->shapes.push_back(e);
  return FPW_OK;
}

int fpw_ctx_clear_shapes(fpw_ctx* ctx) {
  if (!ctx) return FPW_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->shapes.clear();
  return FPW_OK;
}

int fpw_ctx_last_shape(fpw_ctx* ctx, int* threads, int* freqs_per_thread, int* obs_chunk, int* grid) {
  if (!ctx || !threads || !freqs_per_thread || !obs_chunk || !grid) return FPW_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  *threads = ctx->last_shape.threads;
  *freqs_per_thread = ctx->last_shape.R;
  *obs_chunk = ctx->last_shape.obs_chunk;
  *grid = ctx->last_grid;
  return FPW_OK;
}

int fpw_ctx_set_wait_limit(fpw_ctx* ctx, int64_t clocks) {
  if (!ctx || clocks < 0) return FPW_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->wait_clocks = (long long)clocks;
  return FPW_OK;
}

int fpw_ctx_set_timing(fpw_ctx* ctx, int enable) {
  if (!ctx) return FPW_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->timing = enable != 0;
  return FPW_OK;
}

int fpw_ctx_kernel_time(fpw_ctx* ctx, double* ms, int64_t* launches) {
  if (!ctx || !ms || !launches) return FPW_EINVAL;
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  double total = 0.0;
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    FPW_CK(cudaEventSynchronize(ctx->ev[i + 1]));
    float e = 0.f;
    FPW_CK(cudaEventElapsedTime(&e, ctx->ev[i], ctx->ev[i + 1]));
    total += e;
  }
  *ms = total;
  *launches = (int64_t)(ctx->ev_used / 2);
  ctx->ev_used = 0;
  return FPW_OK;
}

int fpw_ctx_status(fpw_ctx* ctx) {
  if (!ctx) return FPW_EINVAL;
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  FPW_CK(cudaStreamSynchronize(ctx->last_stream));
  unsigned w = 0;
  FPW_CK(cudaMemcpy(&w, static_cast<unsigned*>(ctx->words.p) + 2, sizeof(unsigned), cudaMemcpyDeviceToHost));
  FPW_CK(cudaMemset(static_cast<unsigned*>(ctx->words.p) + 2, 0, sizeof(unsigned)));
  return status_to_code(w);
}

int fpw_periodogram_batch_ex(fpw_ctx* ctx, void* stream, const fpw_params* params, const int64_t* offsets,
                             const int64_t* offsets_host, int64_t ncurves, const double* t, const double* x,
                             const double* sigma, const double* freqs, int64_t nfreq, int M, int k,
                             int32_t* topk_idx, float* topk_S, double* S_out) {
  if (!ctx || ncurves < 0 || nfreq < 0 || M < 1 || k < 0 || k > FPW_MAX_TOPK) return FPW_EINVAL;
  if (ncurves > 0 && k > 0 && (!topk_idx || !topk_S)) return FPW_EINVAL;
  return batch_entry(ctx, stream, params, offsets, offsets_host, ncurves, t, x, sigma, freqs, nfreq, M, k, topk_idx,
                     topk_S, S_out, nullptr, 0, 0);
}

int fpw_periodogram_batch_bins(fpw_ctx* ctx, void* stream, const fpw_params* params, const int64_t* offsets,
                               const int64_t* offsets_host, int64_t ncurves, const double* t, const double* x,
                               const double* sigma, const double* freqs, int64_t nfreq, int M, int64_t k0, int64_t k1,
                               int32_t* bins_out, double* S_out) {
  if (!ctx || ncurves < 0 || nfreq < 0 || M < 1 || k0 < 0 || k1 < k0 || k1 > nfreq) return FPW_EINVAL;
  if (ncurves > 0 && k1 > k0 && !bins_out) return FPW_EINVAL;
  return batch_entry(ctx, stream, params, offsets, offsets_host, ncurves, t, x, sigma, freqs, nfreq, M, 0, nullptr,
                     nullptr, S_out, k1 > k0 ? bins_out : nullptr, k0, k1);
}

int fpw_periodogram_batch_multi(fpw_ctx* ctx, void* stream, const fpw_params* params, const int64_t* offsets,
                                const int64_t* offsets_host, int64_t ncurves, const double* t, const double* x,
                                const double* sigma, const double* freqs, int64_t nfreq, int M_max, const int* groups,
                                int ngroups, int k, int32_t* topk_idx, int32_t* topk_offset, float* topk_S,
                                double* S_out) {
  if (!ctx || ncurves < 0 || nfreq < 0 || M_max < 1 || k < 0 || k > FPW_MAX_TOPK) return FPW_EINVAL;
  if (!groups || ngroups < 1 || ngroups > kMaxGroups) return FPW_EINVAL;
  for (int q = 0; q < ngroups; ++q)
    if (groups[q] < 1 || groups[q] > 64 || M_max % groups[q] != 0) return FPW_EINVAL;
  if (k > 0 && nfreq >= ((int64_t)1 << 25)) return FPW_EINVAL;  // ranking key (k << 6) | offset must fit 31 bits
  if (ncurves > 0 && !offsets) return FPW_EINVAL;
  if (ncurves > 0 && nfreq > 0 && !freqs) return FPW_EINVAL;
  if (ncurves > 0 && k > 0 && (!topk_idx || !topk_S || !topk_offset)) return FPW_EINVAL;
  fpw_params p;
  fpw_params_default(&p);
  if (params) p = *params;
  if (!valid_params(p)) return FPW_EINVAL;
  if (p.accum != FPW_ACCUM_FP32 || p.phase_mode == FPW_PHASE_FP64) return FPW_ENOTSUP;
  if (p.threads > 256) return FPW_ENOTSUP;  // the several-M kernel's launch bound
  DeviceGuard g(ctx->device);
  if (!g.ok) return FPW_ECUDA;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_stale_error();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ctx->last_stream = st;
  if (ncurves == 0) return FPW_OK;
  const int64_t* off_h = offsets_host;
  if (!off_h) {
    ctx->off_host.resize((size_t)ncurves + 1);
    FPW_CK(cudaMemcpyAsync(ctx->off_host.data(), offsets, sizeof(int64_t) * (size_t)(ncurves + 1),
                           cudaMemcpyDeviceToHost, st));
    FPW_CK(cudaStreamSynchronize(st));
    off_h = ctx->off_host.data();
  }
  if (check_offsets(off_h, ncurves) != FPW_OK) return FPW_EINVAL;
  if (off_h[ncurves] > 0 && (!t || !x || !sigma)) return FPW_EINVAL;
  BatchCall b{};
  b.stream = st;
  b.p = p;
  b.offsets = offsets;
  b.off_h = off_h;
  b.C = ncurves;
  b.t = t;
  b.x = x;
  b.sigma = sigma;
  b.freqs = freqs;
  b.F = nfreq;
  b.M = M_max;
  b.k = k;
  b.topk_idx = topk_idx;
  b.topk_S = topk_S;
  b.S_out = S_out;
  b.ngroups = ngroups;
  for (int q = 0; q < ngroups; ++q) b.groups[q] = groups[q];
  b.topk_off = topk_offset;
  if (nfreq == 0) {
    if (k > 0) {
      FPW_CK(launch_fill_topk(topk_idx, topk_S, ncurves * ngroups * k, st));
      FPW_CK(launch_fill_topk(topk_offset, topk_S, ncurves * ngroups * k, st));
    }
    return FPW_OK;
  }
  if (nfreq > ((int64_t)1 << 31) - 1024 || ncurves > ((int64_t)1 << 31) - 1) return FPW_EINVAL;
  return run_tile_path(ctx, b);
}

int fpw_periodogram_batch(const int64_t* offsets, int64_t ncurves, const double* t, const double* x,
                          const double* sigma, const double* freqs, int64_t nfreq, int M, int k, int32_t* topk_idx,
                          float* topk_S) {
  int rc = FPW_OK;
  fpw_ctx* ctx = default_ctx(&rc);
  if (!ctx) return rc;
  rc = fpw_periodogram_batch_ex(ctx, nullptr, nullptr, offsets, nullptr, ncurves, t, x, sigma, freqs, nfreq, M, k,
                                topk_idx, topk_S, nullptr);
  if (rc != FPW_OK) return rc;
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  return sync_status(ctx, nullptr, rc);
}

int fpw_periodogram_ex(fpw_ctx* ctx, void* stream, const fpw_params* params, const double* t, const double* x,
                       const double* sigma, int64_t n, const double* freqs, int64_t nfreq, int M, double* S_out) {
  if (!ctx || n < 0 || nfreq < 0 || M < 1) return FPW_EINVAL;
  if (nfreq > 0 && (!freqs || !S_out)) return FPW_EINVAL;
  if (n > 0 && (!t || !x || !sigma)) return FPW_EINVAL;
  fpw_params p;
  fpw_params_default(&p);
  if (params) p = *params;
  if (!valid_params(p)) return FPW_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return FPW_ECUDA;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_stale_error();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ctx->last_stream = st;
  int64_t off_h[2] = {0, n};
  BatchCall b{};
  b.stream = st;
  b.p = p;
  b.offsets = nullptr;
  b.off_h = off_h;
  b.C = 1;
  b.t = t;
  b.x = x;
  b.sigma = sigma;
  b.freqs = freqs;
  b.F = nfreq;
  b.M = M;
  b.k = 0;
  b.S_out = S_out;
  if (nfreq == 0) return FPW_OK;
  if (p.phase_mode == FPW_PHASE_FP64) {
    // single curve: the plain kernel reads the curve directly
    if (plain_smem_bytes(M) > (size_t)ctx->smem_optin) return FPW_ENOTSUP;
    unsigned* words = static_cast<unsigned*>(ctx->words.p);
    FPW_CK(cudaMemsetAsync(words, 0, 2 * sizeof(unsigned), st));
    FPW_CK(ensure(ctx->curve_bad, 16));
    PrepArgs pa{};
    pa.t = t;
    pa.x = x;
    pa.sigma = sigma;
    pa.ncurves = 1;
    pa.nobs = n;
    pa.freqs = freqs;
    pa.nfreq = nfreq;
    pa.curve_bad = static_cast<uint8_t*>(ctx->curve_bad.p);
    pa.status = words + 1;
    FPW_CK(launch_prep(pa, st));
    PlainArgs a{};
    a.t = t;
    a.x = x;
    a.sigma = sigma;
    a.n = n;
    a.freqs = freqs;
    a.nfreq = nfreq;
    a.M = M;
    a.inv_alpha2 = p.inv_alpha2;
    a.S_out = S_out;
    a.status = words + 1;
    FPW_CK(launch_plain(a, st));
    FPW_CK(launch_latch(words, st));
    return FPW_OK;
  }
  return batch_impl(ctx, b);
}

int fpw_periodogram(const double* t, const double* x, const double* sigma, int64_t n, const double* freqs,
                    int64_t nfreq, int M, double* S_out) {
  int rc = FPW_OK;
  fpw_ctx* ctx = default_ctx(&rc);
  if (!ctx) return rc;
  rc = fpw_periodogram_ex(ctx, nullptr, nullptr, t, x, sigma, n, freqs, nfreq, M, S_out);
  if (rc != FPW_OK) return rc;
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  return sync_status(ctx, nullptr, rc);
}

int fpw_periodogram_batch_host(fpw_ctx* ctx, const fpw_params* params, const int64_t* offsets, int64_t ncurves,
                               const double* t, const double* x, const double* sigma, const double* freqs,
                               int64_t nfreq, int M, int k, int32_t* topk_idx, float* topk_S) {
  if (!ctx || ncurves < 0 || nfreq < 0 || M < 1 || k < 0 || k > FPW_MAX_TOPK) return FPW_EINVAL;
  if (ncurves == 0) return FPW_OK;
  if (!offsets || (nfreq > 0 && !freqs) || (k > 0 && (!topk_idx || !topk_S))) return FPW_EINVAL;
  if (check_offsets(offsets, ncurves) != FPW_OK) return FPW_EINVAL;
  const int64_t nobs = offsets[ncurves];
  if (nobs > 0 && (!t || !x || !sigma)) return FPW_EINVAL;
  cudaStream_t st = nullptr;
  {
    DeviceGuard g(ctx->device);
    if (!g.ok) return FPW_ECUDA;
    std::lock_guard<std::mutex> lk(ctx->mu);
    st = ctx->own_stream;
    FPW_CK(ensure(ctx->h_off, sizeof(int64_t) * (size_t)(ncurves + 1)));
    FPW_CK(ensure(ctx->h_t, sizeof(double) * (size_t)std::max<int64_t>(nobs, 1)));
    FPW_CK(ensure(ctx->h_x, sizeof(double) * (size_t)std::max<int64_t>(nobs, 1)));
    FPW_CK(ensure(ctx->h_sigma, sizeof(double) * (size_t)std::max<int64_t>(nobs, 1)));
    FPW_CK(ensure(ctx->h_freqs, sizeof(double) * (size_t)std::max<int64_t>(nfreq, 1)));
    FPW_CK(ensure(ctx->h_idx, sizeof(int32_t) * (size_t)std::max<int64_t>(ncurves * k, 1)));
    FPW_CK(ensure(ctx->h_S, sizeof(float) * (size_t)std::max<int64_t>(ncurves * k, 1)));
    FPW_CK(cudaMemcpyAsync(ctx->h_off.p, offsets, sizeof(int64_t) * (size_t)(ncurves + 1), cudaMemcpyHostToDevice, st));
    if (nobs > 0) {
      FPW_CK(cudaMemcpyAsync(ctx->h_t.p, t, sizeof(double) * (size_t)nobs, cudaMemcpyHostToDevice, st));
      FPW_CK(cudaMemcpyAsync(ctx->h_x.p, x, sizeof(double) * (size_t)nobs, cudaMemcpyHostToDevice, st));
      FPW_CK(cudaMemcpyAsync(ctx->h_sigma.p, sigma, sizeof(double) * (size_t)nobs, cudaMemcpyHostToDevice, st));
    }
    if (nfreq > 0)
      FPW_CK(cudaMemcpyAsync(ctx->h_freqs.p, freqs, sizeof(double) * (size_t)nfreq, cudaMemcpyHostToDevice, st));
  }
  int rc = fpw_periodogram_batch_ex(ctx, st, params, static_cast<const int64_t*>(ctx->h_off.p), offsets, ncurves,
                                    static_cast<const double*>(ctx->h_t.p), static_cast<const double*>(ctx->h_x.p),
                                    static_cast<const double*>(ctx->h_sigma.p),
                                    static_cast<const double*>(ctx->h_freqs.p), nfreq, M, k,
                                    static_cast<int32_t*>(ctx->h_idx.p), static_cast<float*>(ctx->h_S.p), nullptr);
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (rc != FPW_OK) {
    cudaStreamSynchronize(st);
    return rc;
  }
  if (k > 0) {
    FPW_CK(cudaMemcpyAsync(topk_idx, ctx->h_idx.p, sizeof(int32_t) * (size_t)(ncurves * k), cudaMemcpyDeviceToHost, st));
    FPW_CK(cudaMemcpyAsync(topk_S, ctx->h_S.p, sizeof(float) * (size_t)(ncurves * k), cudaMemcpyDeviceToHost, st));
  }
  return sync_status(ctx, st, FPW_OK);
}

int fpw_periodogram_shared(fpw_ctx* ctx, void* stream, const fpw_params* params, const double* t, int64_t n,
                           int64_t ncurves, const double* x, const double* sigma, const double* freqs, int64_t nfreq,
                           int M, int k, int32_t* topk_idx, float* topk_S, double* S_out) {
  if (!ctx || n < 0 || ncurves < 0 || nfreq < 0 || M < 1 || k < 0 || k > FPW_MAX_TOPK) return FPW_EINVAL;
  if (ncurves > 0 && nfreq > 0 && !freqs) return FPW_EINVAL;
  if (ncurves > 0 && n > 0 && (!t || !x || !sigma)) return FPW_EINVAL;
  if (ncurves > 0 && k > 0 && (!topk_idx || !topk_S)) return FPW_EINVAL;
  if (nfreq > ((int64_t)1 << 31) - 1024 || ncurves > ((int64_t)1 << 31) - 1) return FPW_EINVAL;
  fpw_params p;
  fpw_params_default(&p);
  if (params) p = *params;
  if (!valid_params(p)) return FPW_EINVAL;
  if (p.phase_mode != FPW_PHASE_FIXED64 || p.accum != FPW_ACCUM_FP32) return FPW_ENOTSUP;
  int n_mma = 0;
  const int fpm = shared_freqs_per_mma(M, &n_mma);
  if (fpm == 0) return FPW_ENOTSUP;
  DeviceGuard g(ctx->device);
  if (!g.ok) return FPW_ECUDA;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_stale_error();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ctx->last_stream = st;
  if ((size_t)ctx->smem_optin < shared_smem_bytes()) return FPW_ENOTSUP;
  if (ncurves == 0) return FPW_OK;
  unsigned* words = static_cast<unsigned*>(ctx->words.p);
  if (nfreq == 0) {
    if (k > 0) FPW_CK(launch_fill_topk(topk_idx, topk_S, ncurves * k, st));
    return FPW_OK;
  }
  const int64_t per = shared_curves_per_group();
  SharedArgs a{};
  a.t = t;
  a.n = n;
  a.ncurves = ncurves;
  a.x = x;
  a.sigma = sigma;
  a.freqs = freqs;
  a.nfreq = nfreq;
  a.M = M;
  a.fpm = fpm;
  a.n_mma = n_mma;
  a.npass = (nfreq + 2 * fpm - 1) / (2 * fpm);
  a.ngroups = (ncurves + per - 1) / per;
  a.nchunks = (n + 31) / 32;
  a.inv_alpha2 = p.inv_alpha2;
  a.k = k;
  a.peak_raw = p.peak_mode == FPW_PEAK_RAW ? 1 : 0;
  a.topk_idx = topk_idx;
  a.topk_S = topk_S;
  a.S_out = S_out;
  FPW_CK(ensure(ctx->sh_image, std::max<size_t>(shared_image_bytes(ncurves, n), 256)));
  FPW_CK(ensure(ctx->sh_scale, (size_t)(a.ngroups * per) * 2 * sizeof(float)));
  FPW_CK(ensure(ctx->sh_step, sizeof(unsigned long long) * (size_t)(n + 1)));
  FPW_CK(ensure(ctx->sh_sink, 32 * 64 * (sizeof(float) + sizeof(double))));
  FPW_CK(ensure(ctx->curve_bad, (size_t)(a.ngroups * per) + 16));
  if (k > 0) FPW_CK(ensure(ctx->sh_S32, (size_t)ncurves * (size_t)nfreq * sizeof(float)));
  a.image = static_cast<unsigned char*>(ctx->sh_image.p);
  a.inv_scale = static_cast<float*>(ctx->sh_scale.p);
  a.step = static_cast<unsigned long long*>(ctx->sh_step.p);
  a.scratch64 = static_cast<double*>(ctx->sh_sink.p);
  a.scratch32 = reinterpret_cast<float*>(a.scratch64 + 32 * 64);
  a.tmax_bits = reinterpret_cast<unsigned long long*>(static_cast<unsigned*>(ctx->words.p) + 8);
  a.curve_bad = static_cast<uint8_t*>(ctx->curve_bad.p);
  a.S32 = k > 0 ? static_cast<float*>(ctx->sh_S32.p) : nullptr;
  a.status = words + 1;
  a.wait_clocks = ctx->wait_clocks;
  if (ctx->timing) {
    while (ctx->ev.size() < ctx->ev_used + 2) {
      cudaEvent_t e;
      FPW_CK(cudaEventCreate(&e));
      ctx->ev.push_back(e);
    }
    a.timing_start = ctx->ev[ctx->ev_used];
    a.timing_stop = ctx->ev[ctx->ev_used + 1];
    ctx->ev_used += 2;
  }
  FPW_CK(cudaMemsetAsync(words, 0, 2 * sizeof(unsigned), st));
  FPW_CK(launch_shared(a, ctx->nsm, st));
  FPW_CK(launch_latch(words, st));
  return FPW_OK;
}

int fpw_periodogram_drift(fpw_ctx* ctx, void* stream, const fpw_params* params, const int64_t* offsets,
                          int64_t ncurves, const double* t, const double* x, const double* sigma, const double* freqs,
                          int64_t nfreq, int M, int K, double beta, int k, int32_t* topk_idx, float* topk_S,
                          double* S_out) {
  if (!ctx || ncurves < 0 || nfreq < 0 || M < 1 || k < 0 || k > FPW_MAX_TOPK) return FPW_EINVAL;
  if (K < 0 || K > drift_max_basis() || !(beta >= 0.0) || !std::isfinite(beta)) return FPW_EINVAL;
  if (ncurves > 0 && (!offsets || (nfreq > 0 && !freqs))) return FPW_EINVAL;
  if (ncurves > 0 && k > 0 && (!topk_idx || !topk_S)) return FPW_EINVAL;
  if (nfreq > ((int64_t)1 << 31) - 1024 || ncurves > 65535) return FPW_EINVAL;
  fpw_params p;
  fpw_params_default(&p);
  if (params) p = *params;
  if (!valid_params(p)) return FPW_EINVAL;
  if (p.phase_mode != FPW_PHASE_FIXED64 || p.accum != FPW_ACCUM_FP32) return FPW_ENOTSUP;
  DeviceGuard g(ctx->device);
  if (!g.ok) return FPW_ECUDA;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_stale_error();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ctx->last_stream = st;
  // threads (32..128) and frequencies per thread (1 or 2) from params when
  // set; by default the largest block with one frequency per thread, and two
  // frequencies per thread for K <= 1 where they fit (8-byte bins: measured
  // 16 % faster at K = 0; slower from K = 2 on, where 16-byte bins halve the
  // resident warps)
  if (p.threads != 0 && (p.threads % 32 != 0 || p.threads < 32 || p.threads > 128)) return FPW_ENOTSUP;
  if (p.freqs_per_thread != 0 && p.freqs_per_thread != 1 && p.freqs_per_thread != 2) return FPW_ENOTSUP;
  const int T = p.threads != 0 ? p.threads : drift_threads(M, K, ctx->smem_optin);
  if (T == 0 || !drift_fits(M, K, T, 1, ctx->smem_optin)) return FPW_ENOTSUP;
  int R = p.freqs_per_thread;
  if (R == 0) R = (K <= 1 && drift_fits(M, K, T, 2, ctx->smem_optin)) ? 2 : 1;
  if (!drift_fits(M, K, T, R, ctx->smem_optin)) return FPW_ENOTSUP;
  if (ncurves == 0) return FPW_OK;
  // every offset is checked before a kernel indexes the observations with it
  ctx->off_host.resize((size_t)ncurves + 1);
  FPW_CK(cudaMemcpyAsync(ctx->off_host.data(), offsets, sizeof(int64_t) * (size_t)(ncurves + 1),
                         cudaMemcpyDeviceToHost, st));
  FPW_CK(cudaStreamSynchronize(st));
  if (check_offsets(ctx->off_host.data(), ncurves) != FPW_OK) return FPW_EINVAL;
  const int64_t nobs = ctx->off_host[(size_t)ncurves];
  if (nobs > 0 && (!t || !x || !sigma)) return FPW_EINVAL;
  unsigned* words = static_cast<unsigned*>(ctx->words.p);
  if (nfreq == 0) {
    if (k > 0) FPW_CK(launch_fill_topk(topk_idx, topk_S, ncurves * k, st));
    return FPW_OK;
  }
  FPW_CK(ensure(ctx->dr_payload, drift_payload_bytes() * (size_t)std::max<int64_t>(nobs, 1)));
  FPW_CK(ensure(ctx->dr_H0, sizeof(double) * 16 * (size_t)ncurves));
  FPW_CK(ensure(ctx->dr_g, sizeof(double) * 4 * (size_t)ncurves));
  FPW_CK(ensure(ctx->dr_tabs, sizeof(double) * (size_t)ncurves));
  FPW_CK(ensure(ctx->curve_bad, (size_t)ncurves + 16));
  if (k > 0) FPW_CK(ensure(ctx->sh_S32, (size_t)ncurves * (size_t)nfreq * sizeof(float)));
  DriftArgs a{};
  a.offsets = offsets;
  a.ncurves = ncurves;
  a.t = t;
  a.x = x;
  a.sigma = sigma;
  a.freqs = freqs;
  a.nfreq = nfreq;
  a.M = M;
  a.K = K;
  a.beta = beta;
  a.inv_alpha2 = p.inv_alpha2;
  a.payload = ctx->dr_payload.p;
  a.tabs = static_cast<double*>(ctx->dr_tabs.p);
  a.H0 = static_cast<double*>(ctx->dr_H0.p);
  a.g = static_cast<double*>(ctx->dr_g.p);
  a.curve_bad = static_cast<uint8_t*>(ctx->curve_bad.p);
  a.status = words + 1;
  a.S32 = k > 0 ? static_cast<float*>(ctx->sh_S32.p) : nullptr;
  a.S_out = S_out;
  a.k = k;
  a.peak_raw = p.peak_mode == FPW_PEAK_RAW ? 1 : 0;
  a.topk_idx = topk_idx;
  a.topk_S = topk_S;
  if (ctx->timing) {
    while (ctx->ev.size() < ctx->ev_used + 2) {
      cudaEvent_t e;
      FPW_CK(cudaEventCreate(&e));
      ctx->ev.push_back(e);
    }
    a.timing_start = ctx->ev[ctx->ev_used];
    a.timing_stop = ctx->ev[ctx->ev_used + 1];
    ctx->ev_used += 2;
  }
  FPW_CK(cudaMemsetAsync(words, 0, 2 * sizeof(unsigned), st));
  FPW_CK(launch_drift(a, T, R, st));
  FPW_CK(launch_latch(words, st));
  return FPW_OK;
}

int fpw_phase_entropy(fpw_ctx* ctx, void* stream, const double* t, int64_t n, const double* freqs, int64_t nfreq,
                      int M, float* H_out) {
  if (!ctx || n < 0 || nfreq < 0 || M < 1 || M > 256) return FPW_EINVAL;
  if (nfreq > 0 && (!freqs || !H_out)) return FPW_EINVAL;
  if (n > 0 && !t) return FPW_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return FPW_ECUDA;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_stale_error();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ctx->last_stream = st;
  FPW_CK(launch_entropy_dense(t, n, freqs, nfreq, M, H_out, st));
  return FPW_OK;
}

int fpw_phase_entropy_peaks(fpw_ctx* ctx, void* stream, const int64_t* offsets, int64_t ncurves, const double* t,
                            const double* freqs, int64_t nfreq, int M, int k, const int32_t* topk_idx, float* H_out,
                            float* z_out) {
  if (!ctx || ncurves < 0 || nfreq < 0 || M < 1 || M > 4096 || k < 0) return FPW_EINVAL;
  if (ncurves > 0 && k > 0 && (!offsets || !freqs || !topk_idx || !H_out || !z_out || !t)) return FPW_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return FPW_ECUDA;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_stale_error();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ctx->last_stream = st;
  FPW_CK(launch_entropy_peaks(offsets, ncurves, t, freqs, nfreq, M, k, topk_idx, H_out, z_out, st));
  return FPW_OK;
}

}  // extern "C"
