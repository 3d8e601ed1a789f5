// api.cu -- the C ABI of libskipper (declared in include/skipper.h).
//
// Host side only: argument checks, scratch ownership, kernel launches on the
// caller's stream, the batched CUDA graph, the autotuner and error reporting.
// Every step of the matching itself runs in the kernels of sweep.cu and
// check.cu; there is no host fallback.
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <cuda_runtime.h>

#include "internal.h"
#include "skipper.h"

using namespace skp;

namespace {

thread_local char g_err[512] = "";

mm_status fail(mm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

#define CUDA_TRY(expr)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA, "%s: %s (%s)", \
                  #expr, cudaGetErrorString(e_), __func__);                                  \
  } while (0)

constexpr uint32_t kDefaultGrain = 2048;   // partition table sized at creation for this grain
constexpr int kDefaultBlock = 512;
constexpr uint64_t kDefaultSpin = 1ull << 20;

struct BatchGraph {
  bool valid = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t n_plan = nullptr, n_prepare = nullptr, n_sweep = nullptr, n_pairs = nullptr,
                  n_copy = nullptr;
  // signature of the options the graph was built for
  uint32_t status_bits = 0, serial = 0, grain = 0, block = 0, blocks_per_sm = 0, wpg = 0;
  bool sym = false;
  bool with_pairs = false;
  uint64_t num_graphs = 0;
};

}  // namespace

void skp::set_error_message(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

struct mm_graph {
  int device = 0;
  int num_sms = 0;
  int l2_bytes = 0;                   // the device's L2 size
  uint64_t n = 0, nnz = 0;            // nnz: stored entries (CSR) or listed edges (edge list)
  bool coo = false;                   // made by mm_create_coo: an edge list, no CSR
  bool host_mapped = false;           // the input arrays are host memory read in place
  const int64_t* offsets = nullptr;
  const uint32_t* nbrs = nullptr;
  const uint32_t* src = nullptr;      // edge list (coo): edge i = (src[i], dst[i])
  const uint32_t* dst = nullptr;
  uint32_t* state = nullptr;          // ceil(n/4) words (+ slack)
  int64_t* part = nullptr;
  uint64_t part_units_cap = 0;
  unsigned long long* ctrl = nullptr;  // [0] work counter, [1] err word, [2] csr-check count,
                                       // [8..16] checker counters
  uint32_t* seen_bits = nullptr;
  unsigned long long* stats = nullptr;  // sweep statistics, allocated on first stats call
  bool stats_valid = false;
  int last_bits = 0;                   // layout and state array of the last mm_skipper call
  const uint32_t* last_state = nullptr;
  unsigned char* found = nullptr;      // checker scratch, allocated on first mm_validate
  int64_t* check_part = nullptr;
  uint64_t* tile_counts = nullptr;
  uint64_t tile_cap = 0;
  uint32_t* h_err = nullptr;           // pinned
  unsigned long long* h_counters = nullptr;  // pinned, 16 words
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // event sets of timed calls, read back without blocking the calls themselves
  static constexpr uint32_t kHist = 256;
  cudaEvent_t hist[kHist][4] = {};
  uint64_t hist_units[kHist] = {};
  bool hist_compact[kHist] = {};
  uint64_t hist_count = 0;   // timed calls since the last mm_timing_history
  bool hist_ready = false;
  mm_timing timing{};
  BatchGraph bg;
  // batches partitioned per member graph (batch.cu): local ids, warps-per-graph cap
  bool local_ids = false;             // made with MM_BATCH_LOCAL_IDS
  uint64_t state_words = 0;           // words allocated at `state`
  uint64_t* btab = nullptr;           // ubase [G+1] | sbase [G+1] | totals [2]
  uint64_t btab_graphs = 0;
  uint32_t* bgid = nullptr;
  int64_t* bpart = nullptr;
  uint64_t bunits_cap = 0;
  BatchGraph bg2;                     // the CUDA graph of these launches
  // mm_skipper_to_host: the stream of the copies back, one event per launch,
  // pinned unit starts [0, MM_MAX_PIECES] and row splits after them
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t piece_ev[MM_MAX_PIECES + 1] = {};
  cudaEvent_t pieces_done = nullptr;  // the last call's work, so its pinned reads are over
  uint64_t* h_split = nullptr;
};

namespace {

unsigned long long* work_ptr(mm_graph* g) { return g->ctrl; }
uint32_t* err_ptr(mm_graph* g) { return reinterpret_cast<uint32_t*>(g->ctrl + 1); }
unsigned long long* csr_bad_ptr(mm_graph* g) { return g->ctrl + 2; }
unsigned long long* counters_ptr(mm_graph* g) { return g->ctrl + 8; }

struct Resolved {
  int bits;   // state layout: 2, 8 (packed fields) or 32 (word = mate)
  bool word;
  bool serial;
  uint32_t grain;
  int block;
  int blocks_per_sm;
  bool nosync, timing, use_graph, l2_persist, stats, sym, sel, stage;
  uint32_t wpg;
  bool lean;          // the 32-register instance of the plain / symmetric sweep
  bool disperse;      // units handed out in dispersed runs
  uint64_t spin_limit, poison;
};

mm_status resolve(const mm_graph* g, const mm_options* o, Resolved* r) {
  mm_options d;
  mm_default_options(&d);
  if (!o) o = &d;
  const uint32_t bits = o->status_bits ? o->status_bits : 8u;
  if (bits != 2 && bits != 8 && bits != 32)
    return fail(MM_ERR_ARG, "status_bits must be 2, 8 or 32 (got %u)", bits);
  r->bits = (int)bits;
  r->word = bits == 32;
  r->serial = o->serial != 0;
  r->grain = o->grain;
  if (r->grain % 128 || r->grain > (1u << 24))
    return fail(MM_ERR_ARG, "grain must be a multiple of 128 and at most 2^24 (got %u)", r->grain);
  r->block = o->block_threads ? (int)o->block_threads : kDefaultBlock;
  if (r->block < 32 || r->block > 512 || r->block % 32)
    return fail(MM_ERR_ARG, "block_threads must be a multiple of 32 in [32, 512] (got %d)", r->block);
  r->blocks_per_sm = (int)o->blocks_per_sm;
  r->nosync = o->nosync != 0;
  r->timing = o->timing != 0;
  r->use_graph = o->use_graph != 0;
  r->l2_persist = o->l2_persist != 0;
  r->stats = o->stats != 0;
  r->sym = o->symmetric != 0;
  if (o->id_loads > MM_ID_LOADS_SELECTIVE) return fail(MM_ERR_ARG, "id_loads must be 0, 1 or 2 (got %u)", o->id_loads);
  r->sel = o->id_loads == MM_ID_LOADS_SELECTIVE || (o->id_loads == MM_ID_LOADS_AUTO && g->host_mapped);
  r->stage = o->stage_windows != 0;
  r->wpg = o->warps_per_graph;
  // defaults by the state array's size: at most half the L2 -> 64 warps per
  // SM and dispersed units; larger -> 48 warps per SM and ascending units
  const uint64_t state_bytes = r->word ? 4 * g->n : 4 * packed_words(g->n, r->bits);
  const bool fits = g->l2_bytes > 0 && 2 * state_bytes <= (uint64_t)g->l2_bytes;
  r->lean = sweep_lean(r->bits, r->block, r->blocks_per_sm, fits);
  if (o->unit_order > MM_ORDER_DISPERSED) return fail(MM_ERR_ARG, "unit_order must be 0, 1 or 2 (got %u)", o->unit_order);
  r->disperse = o->unit_order == MM_ORDER_DISPERSED || (o->unit_order == MM_ORDER_AUTO && fits);
  // grain 0: about two units per resident warp, the nearest power of two in
  // [512, 8192] -- small graphs need many units to occupy the GPU, large ones
  // lose to per-unit set-up below 4096; over the host link, where every
  // unit's first window waits on the link, up to 32768
  if (r->grain == 0) {
    const uint64_t items = g->coo ? g->nnz : g->n + g->nnz;
    const uint64_t warps = (uint64_t)(g->num_sms > 0 ? g->num_sms : 1) * (r->lean ? 64u : 48u);
    const uint64_t target = items / (2 * warps);
    const uint32_t cap = g->host_mapped ? 32768u : 8192u;
    uint32_t grain = 512;
    while (grain < cap && (uint64_t)grain * 1414 < target * 1000) grain *= 2;
    r->grain = grain;
  }
  r->spin_limit = o->spin_limit ? o->spin_limit : kDefaultSpin;
  r->poison = o->poison_vertex;
  if (r->poison > g->n) return fail(MM_ERR_ARG, "poison_vertex out of range");
  if (r->word && g->n > MM_MAX_VERTICES && !g->local_ids) return fail(MM_ERR_ARG, "n too large for 32-bit states");
  return MM_OK;
}

mm_status ensure_part(mm_graph* g, uint64_t units) {
  if (units <= g->part_units_cap && g->part) return MM_OK;
  if (g->part) cudaFree(g->part);
  g->part = nullptr;
  g->part_units_cap = 0;
  CUDA_TRY(cudaMalloc(&g->part, (units + 1) * 2 * sizeof(int64_t)));
  g->part_units_cap = units;
  return MM_OK;
}

// the persistent grid of a CSR sweep; `lean`: the 32-register instance runs
int sweep_grid(const mm_graph* g, const Resolved& r, bool lean) {
  const int per_sm = r.blocks_per_sm > 0 ? r.blocks_per_sm : sweep_blocks_per_sm(r.bits, r.block, lean);
  return g->num_sms * per_sm;
}

int prepare_grid(const mm_graph* g) { return g->num_sms * 8; }

// Grids of one mm_skipper call sized to its graph: a small graph gets only the
// blocks it can use (its units for the sweep, its fills and units for the
// preparation), so a call on a 1k-edge graph does not launch a full
// persistent grid.
int prepare_grid_for(const mm_graph* g, uint64_t units) {
  const uint64_t items = (g->n / 4 + 1 > units + 1 ? g->n / 4 + 1 : units + 1);
  const uint64_t blocks = (items + 255) / 256;
  return blocks < (uint64_t)prepare_grid(g) ? (int)blocks : prepare_grid(g);
}
int sweep_grid_for(const mm_graph* g, const Resolved& r, bool lean, uint64_t units) {
  const uint64_t warps = (uint64_t)(r.block / 32);
  const uint64_t blocks = (units + warps - 1) / warps;
  const int full = sweep_grid(g, r, lean);
  return blocks < (uint64_t)full ? (int)(blocks ? blocks : 1) : full;
}

SweepParams make_params(mm_graph* g, const Resolved& r, uint32_t* d_mate) {
  SweepParams P{};
  P.n = g->n;
  P.nnz = g->nnz;
  P.offsets = g->offsets;
  P.nbrs = g->nbrs;
  P.mate = d_mate;
  P.state = r.word ? d_mate : g->state;
  P.grain = r.grain;
  P.units = (g->n + g->nnz + r.grain - 1) / r.grain;
  P.part = g->part;
  P.work = work_ptr(g);
  P.err = err_ptr(g);
  P.spin_limit = r.spin_limit;
  P.poison = r.poison;
  P.sym = r.sym && !r.serial;
  P.sel = r.sel && !r.serial;
  // staged windows: bulk copies want 16-byte aligned device arrays
  const bool aligned16 = ((reinterpret_cast<uintptr_t>(g->offsets) |
                           reinterpret_cast<uintptr_t>(P.state)) & 15u) == 0;
  P.tile = r.stage && !r.serial && !r.word && !g->host_mapped && aligned16;
  // the 32-register instance exists for the plain and symmetric sweeps only
  P.lean = r.lean && !r.serial && !r.stats && !P.sel && !P.tile;
  P.disperse = r.disperse ? 1u : 0u;
  return P;
}

mm_status read_err(mm_graph* g, cudaStream_t s) {
  CUDA_TRY(cudaStreamSynchronize(s));
  const uint32_t e = *g->h_err;
  if (e & kErrTimeout) return fail(MM_ERR_TIMEOUT, "a wait on a reserved vertex ran past spin_limit");
  if (e & kErrBadId) return fail(MM_ERR_BAD_GRAPH, "a neighbour id >= n was met");
  return MM_OK;
}

// L2 persisting window over the state array for the sweep (opt-in); the
// stream attribute and the context's set-aside are put back afterwards.
struct L2Window {
  bool on = false, limit_set = false;
  cudaStream_t s{};
  size_t old_limit = 0;
  // a call that fails between open and close still puts the stream attribute
  // and the set-aside back (quietly: the call's own error message stands)
  ~L2Window() {
    if (on) {
      cudaStreamAttrValue a{};
      a.accessPolicyWindow.num_bytes = 0;
      cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &a);
      cudaCtxResetPersistingL2Cache();
    }
    if (limit_set) cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
  }
  mm_status open(mm_graph* g, const Resolved& r, cudaStream_t st, const uint32_t* base, size_t bytes) {
    if (!r.l2_persist) return MM_OK;
    int max_win = 0, max_persist = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, g->device));
    CUDA_TRY(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, g->device));
    if (max_win <= 0 || max_persist <= 0) return MM_OK;
    CUDA_TRY(cudaDeviceGetLimit(&old_limit, cudaLimitPersistingL2CacheSize));
    const size_t want = bytes < (size_t)max_persist ? bytes : (size_t)max_persist;
    CUDA_TRY(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want));
    limit_set = true;
    s = st;
    cudaStreamAttrValue a{};
    a.accessPolicyWindow.base_ptr = const_cast<uint32_t*>(base);
    a.accessPolicyWindow.num_bytes = bytes < (size_t)max_win ? bytes : (size_t)max_win;
    a.accessPolicyWindow.hitRatio = a.accessPolicyWindow.num_bytes > want
                                        ? (float)want / (float)a.accessPolicyWindow.num_bytes
                                        : 1.0f;
    a.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    a.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    CUDA_TRY(cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &a));
    on = true;
    return MM_OK;
  }
  mm_status close() {
    if (on) {
      on = false;
      cudaStreamAttrValue a{};
      a.accessPolicyWindow.num_bytes = 0;
      CUDA_TRY(cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &a));
      CUDA_TRY(cudaCtxResetPersistingL2Cache());
    }
    if (limit_set) {
      limit_set = false;
      CUDA_TRY(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit));
    }
    return MM_OK;
  }
};

mm_status ensure_pieces(mm_graph* g) {
  if (g->h_split) return MM_OK;
  CUDA_TRY(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking));
  for (auto& e : g->piece_ev) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&g->pieces_done, cudaEventDisableTiming));
  CUDA_TRY(cudaHostAlloc(&g->h_split, 2 * (MM_MAX_PIECES + 1) * sizeof(uint64_t), cudaHostAllocDefault));
  return MM_OK;
}

mm_status ensure_hist(mm_graph* g) {
  if (g->hist_ready) return MM_OK;
  for (auto& set : g->hist)
    for (auto& e : set) CUDA_TRY(cudaEventCreate(&e));
  g->hist_ready = true;
  return MM_OK;
}

// events of the next timed call (the ring keeps the latest kHist calls)
cudaEvent_t* next_hist(mm_graph* g, uint64_t units, bool compact) {
  const uint32_t slot = (uint32_t)(g->hist_count % mm_graph::kHist);
  g->hist_units[slot] = units;
  g->hist_compact[slot] = compact;
  ++g->hist_count;
  return g->hist[slot];
}

mm_status read_slot(mm_graph* g, uint32_t slot, mm_timing* out) {
  cudaEvent_t* ev = g->hist[slot];
  CUDA_TRY(cudaEventSynchronize(ev[3]));
  float a = 0, b = 0, c = 0, t = 0;
  CUDA_TRY(cudaEventElapsedTime(&a, ev[0], ev[1]));
  CUDA_TRY(cudaEventElapsedTime(&b, ev[1], ev[2]));
  CUDA_TRY(cudaEventElapsedTime(&c, ev[2], ev[3]));
  CUDA_TRY(cudaEventElapsedTime(&t, ev[0], ev[3]));
  *out = mm_timing{};
  out->init_ms = a;
  out->sweep_ms = b;
  out->compact_ms = g->hist_compact[slot] ? c : 0.0f;
  out->total_ms = t;
  out->units = g->hist_units[slot];
  return MM_OK;
}

// MM_HOST_MAPPED: the device address of host memory (page-locked, or any
// host memory on a device that walks the host's page tables; the same address
// under unified addressing); MM_ERR_ARG when the device cannot address it.
template <class T>
mm_status map_host(const T** p, const char* what) {
  void* d = nullptr;
  const cudaError_t e = cudaHostGetDevicePointer(&d, const_cast<T*>(*p), 0);
  if (e != cudaSuccess) {
    cudaGetLastError();  // not sticky; clear it for the caller's next call
    return fail(MM_ERR_ARG, "%s is host memory the device cannot address (MM_HOST_MAPPED): %s",
                what, cudaGetErrorString(e));
  }
  *p = static_cast<const T*>(d);
  return MM_OK;
}

mm_status check_flags_and_device(uint32_t flags) {
  if (flags & ~(MM_CHECK_CSR | MM_HOST_MAPPED | MM_BATCH_LOCAL_IDS)) return fail(MM_ERR_ARG, "unknown flags 0x%x", flags);
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (ndev <= 0) return fail(MM_ERR_CUDA, "no CUDA device");
  return MM_OK;
}

// A handle with the scratch every input form needs: state words (one byte a
// vertex, the widest packed layout), control words, compaction tiles, pinned
// status words and events.  On failure nothing is left allocated.
mm_status new_handle(uint64_t n, uint64_t items, cudaStream_t s, mm_graph** out) {
  mm_graph* g = new (std::nothrow) mm_graph();
  if (!g) return fail(MM_ERR_OOM, "host allocation failed");
  auto step = [&](cudaError_t e, const char* what) {
    if (e == cudaSuccess) return MM_OK;
    mm_destroy(g);
    return fail(e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
  };
  mm_status st;
  if ((st = step(cudaGetDevice(&g->device), "cudaGetDevice")) != MM_OK) return st;
  if ((st = step(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device),
                 "cudaDeviceGetAttribute")) != MM_OK)
    return st;
  if ((st = step(cudaDeviceGetAttribute(&g->l2_bytes, cudaDevAttrL2CacheSize, g->device),
                 "cudaDeviceGetAttribute")) != MM_OK)
    return st;
  g->n = n;
  g->nnz = items;
  const uint64_t words = (n + 3) / 4 + 4;
  if ((st = step(cudaMalloc(&g->state, words * sizeof(uint32_t)), "state")) != MM_OK) return st;
  g->state_words = words;
  if ((st = step(cudaMalloc(&g->ctrl, 32 * sizeof(unsigned long long)), "control words")) != MM_OK) return st;
  if ((st = step(cudaMemsetAsync(g->ctrl, 0, 32 * sizeof(unsigned long long), s), "control words")) != MM_OK)
    return st;
  g->tile_cap = (n + kCompactTile - 1) / kCompactTile + 1;
  if ((st = step(cudaMalloc(&g->tile_counts, g->tile_cap * sizeof(uint64_t)), "tiles")) != MM_OK) return st;
  if ((st = step(cudaMallocHost(&g->h_err, 64), "pinned status")) != MM_OK) return st;
  if ((st = step(cudaMallocHost(&g->h_counters, 16 * sizeof(unsigned long long)), "pinned counters")) != MM_OK)
    return st;
  *g->h_err = 0;
  for (auto& e : g->ev)
    if ((st = step(cudaEventCreate(&e), "events")) != MM_OK) return st;
  *out = g;
  return MM_OK;
}

// Run an input check launched on s (its count of violations in the control
// words) and wait for it; on violations the handle is released and the call
// fails with MM_ERR_BAD_GRAPH (msg takes the count).
mm_status device_check(mm_graph* g, cudaStream_t s, cudaError_t launched, const char* msg) {
  cudaError_t e = launched;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->h_counters, csr_bad_ptr(g), sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    mm_destroy(g);
    return fail(MM_ERR_CUDA, "input check: %s", cudaGetErrorString(e));
  }
  if (g->h_counters[0] != 0) {
    const unsigned long long bad = g->h_counters[0];
    mm_destroy(g);
    return fail(MM_ERR_BAD_GRAPH, msg, bad);
  }
  return MM_OK;
}

mm_status check_handle(const mm_graph* g) {
  if (!g) return fail(MM_ERR_ARG, "null handle");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != g->device) return fail(MM_ERR_ARG, "handle belongs to device %d, current is %d", g->device, dev);
  return MM_OK;
}

// mm_skipper on an edge-list handle: prepare, the edge-list sweep (or its
// serial form), the optional ordered pair list, the status read.
mm_status skipper_coo(mm_graph* g, const Resolved& r, uint32_t* d_mate, uint32_t* d_pairs,
                      uint64_t cap, uint64_t* d_count, cudaStream_t s) {
  mm_status st = MM_OK;
  CooParams C{};
  C.P.n = g->n;
  C.P.nnz = g->nnz;
  C.P.mate = d_mate;
  C.P.state = r.word ? d_mate : g->state;
  C.P.work = work_ptr(g);
  C.P.err = err_ptr(g);
  C.P.spin_limit = r.spin_limit;
  C.P.poison = r.poison;
  C.src = g->src;
  C.dst = g->dst;
  C.m = g->nnz;
  C.grain = r.grain;
  C.units = (g->nnz + r.grain - 1) / r.grain;
  C.vec = ((reinterpret_cast<uintptr_t>(g->src) | reinterpret_cast<uintptr_t>(g->dst)) & 15u) == 0;
  g->stats_valid = false;
  if (r.stats && !r.serial) {
    if (!g->stats) CUDA_TRY(cudaMalloc(&g->stats, kStCount * sizeof(unsigned long long)));
    C.P.stats = g->stats;
    g->stats_valid = true;
  }
  CheckScratch cs{counters_ptr(g), g->seen_bits, g->tile_counts, g->tile_cap, nullptr, nullptr};
  g->last_bits = r.bits;
  g->last_state = C.P.state;
  cudaEvent_t* ev = nullptr;
  if (r.timing) {
    if ((st = ensure_hist(g)) != MM_OK) return st;
    ev = next_hist(g, C.units, d_pairs || d_count);
    CUDA_TRY(cudaEventRecord(ev[0], s));
  }
  CUDA_TRY(launch_coo_prepare(C, r.bits, prepare_grid(g), s));
  if (ev) CUDA_TRY(cudaEventRecord(ev[1], s));
  L2Window win;
  if (!r.serial) {
    const int per_sm = r.blocks_per_sm > 0 ? r.blocks_per_sm : coo_blocks_per_sm(r.bits, r.block);
    if ((st = win.open(g, r, s, C.P.state, r.word ? g->n * 4 : packed_words(g->n, r.bits) * 4)) != MM_OK) return st;
    CUDA_TRY(launch_coo_sweep(C, r.bits, g->num_sms * per_sm, r.block, s));
    if ((st = win.close()) != MM_OK) return st;
  } else {
    CUDA_TRY(launch_coo_serial(C, r.bits, s));
  }
  if (ev) CUDA_TRY(cudaEventRecord(ev[2], s));
  if (d_pairs || d_count) CUDA_TRY(launch_compact(g->n, d_mate, d_pairs, d_pairs ? cap : 0, d_count, cs, s));
  if (ev) CUDA_TRY(cudaEventRecord(ev[3], s));
  CUDA_TRY(cudaMemcpyAsync(g->h_err, err_ptr(g), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (r.nosync) return MM_OK;
  return read_err(g, s);
}

}  // namespace

extern "C" {

const char* mm_version(void) { return "skipper-gb300 0.1 sm_103a"; }

const char* mm_last_error(void) { return g_err; }

mm_status mm_default_options(mm_options* o) {
  if (!o) return fail(MM_ERR_ARG, "null options");
  memset(o, 0, sizeof *o);
  o->status_bits = 8;
  o->grain = 0;
  o->block_threads = kDefaultBlock;
  o->spin_limit = kDefaultSpin;
  return MM_OK;
}

mm_status mm_host_device_address(const void* host, const void** device_out) {
  g_err[0] = 0;
  if (!host || !device_out) return fail(MM_ERR_ARG, "null argument");
  const unsigned char* p = static_cast<const unsigned char*>(host);
  mm_status st = map_host(&p, "host address");
  if (st != MM_OK) return st;
  *device_out = p;
  return MM_OK;
}

mm_status mm_create_coo(uint64_t n, uint64_t m, const uint32_t* d_src, const uint32_t* d_dst,
                        uint32_t flags, void* cuda_stream, mm_graph** out) {
  g_err[0] = 0;
  if (!out) return fail(MM_ERR_ARG, "null out");
  *out = nullptr;
  if (n > MM_MAX_VERTICES) return fail(MM_ERR_ARG, "n = %llu exceeds %llu", (unsigned long long)n, MM_MAX_VERTICES);
  if (m && (!d_src || !d_dst)) return fail(MM_ERR_ARG, "null src / dst with m > 0");
  auto aligned = [&]() {
    if ((reinterpret_cast<uintptr_t>(d_src) | reinterpret_cast<uintptr_t>(d_dst)) & 3u)
      return fail(MM_ERR_ARG, "src and dst must be 4-byte aligned");
    return MM_OK;
  };
  mm_status ms = (flags & MM_HOST_MAPPED) ? MM_OK : aligned();
  if (ms != MM_OK) return ms;
  if ((ms = check_flags_and_device(flags)) != MM_OK) return ms;
  if ((flags & MM_HOST_MAPPED) && m) {  // the device addresses of the caller's page-locked arrays
    ms = map_host(&d_src, "src");
    if (ms == MM_OK) ms = map_host(&d_dst, "dst");
    if (ms == MM_OK) ms = aligned();
    if (ms != MM_OK) return ms;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  mm_graph* g = nullptr;
  if ((ms = new_handle(n, m, s, &g)) != MM_OK) return ms;
  g->coo = true;
  g->host_mapped = (flags & MM_HOST_MAPPED) != 0;
  g->src = d_src;
  g->dst = d_dst;
  if (flags & MM_CHECK_CSR) {
    ms = device_check(g, s, launch_coo_check(n, m, d_src, d_dst, csr_bad_ptr(g), prepare_grid(g), s),
                      "edge-list check failed: %llu endpoint ids >= n");
    if (ms != MM_OK) return ms;
  }
  *out = g;
  return MM_OK;
}

mm_status mm_create_csr(uint64_t n, uint64_t nnz, const int64_t* d_offsets, const uint32_t* d_nbrs,
                        uint32_t flags, void* cuda_stream, mm_graph** out) {
  g_err[0] = 0;
  if (!out) return fail(MM_ERR_ARG, "null out");
  *out = nullptr;
  const bool local = (flags & MM_BATCH_LOCAL_IDS) != 0;
  if (local && (flags & (MM_CHECK_CSR | MM_HOST_MAPPED)))
    return fail(MM_ERR_UNSUPPORTED, "MM_BATCH_LOCAL_IDS takes neither MM_CHECK_CSR nor MM_HOST_MAPPED");
  const uint64_t max_n = local ? MM_MAX_BATCH_VERTICES : MM_MAX_VERTICES;
  if (n > max_n) return fail(MM_ERR_ARG, "n = %llu exceeds %llu", (unsigned long long)n, (unsigned long long)max_n);
  if (!d_offsets) return fail(MM_ERR_ARG, "null offsets");
  if (nnz && !d_nbrs) return fail(MM_ERR_ARG, "null nbrs with nnz > 0");
  auto aligned = [&]() {
    if (nnz && (reinterpret_cast<uintptr_t>(d_nbrs) & 15u))
      return fail(MM_ERR_ARG, "nbrs must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(d_offsets) & 7u) return fail(MM_ERR_ARG, "offsets must be 8-byte aligned");
    return MM_OK;
  };
  mm_status ms = (flags & MM_HOST_MAPPED) ? MM_OK : aligned();
  if (ms != MM_OK) return ms;
  if ((ms = check_flags_and_device(flags)) != MM_OK) return ms;
  if (flags & MM_HOST_MAPPED) {  // the device addresses of the caller's page-locked arrays
    ms = map_host(&d_offsets, "offsets");
    if (ms == MM_OK && nnz) ms = map_host(&d_nbrs, "nbrs");
    if (ms == MM_OK) ms = aligned();
    if (ms != MM_OK) return ms;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  mm_graph* g = nullptr;
  if ((ms = new_handle(n, nnz, s, &g)) != MM_OK) return ms;
  g->offsets = d_offsets;
  g->nbrs = d_nbrs;
  g->host_mapped = (flags & MM_HOST_MAPPED) != 0;
  g->local_ids = local;
  if ((ms = ensure_part(g, (n + nnz + kDefaultGrain - 1) / kDefaultGrain)) != MM_OK) {
    mm_destroy(g);
    return ms;
  }
  if (flags & MM_CHECK_CSR) {
    ms = device_check(g, s, launch_csr_check(n, nnz, d_offsets, d_nbrs, csr_bad_ptr(g), prepare_grid(g), s),
                      "CSR check failed: %llu violations (offsets[0] = 0, non-decreasing, "
                      "offsets[n] = nnz, ids < n)");
    if (ms != MM_OK) return ms;
  }
  *out = g;
  return MM_OK;
}

mm_status mm_skipper(mm_graph* g, const mm_options* o, uint32_t* d_mate, uint32_t* d_pairs,
                     uint64_t cap, uint64_t* d_count, void* cuda_stream) {
  g_err[0] = 0;
  mm_status st = check_handle(g);
  if (st != MM_OK) return st;
  if (g->local_ids) return fail(MM_ERR_UNSUPPORTED, "a MM_BATCH_LOCAL_IDS handle runs batched calls only");
  if (!d_mate && g->n) return fail(MM_ERR_ARG, "null mate");
  if (d_pairs && !cap) return fail(MM_ERR_ARG, "pairs given with cap = 0");
  Resolved r;
  if ((st = resolve(g, o, &r)) != MM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (g->coo) return skipper_coo(g, r, d_mate, d_pairs, cap, d_count, s);
  const uint64_t units = (g->n + g->nnz + r.grain - 1) / r.grain;
  if ((st = ensure_part(g, units)) != MM_OK) return st;
  SweepParams P = make_params(g, r, d_mate);
  g->stats_valid = false;
  if (r.stats && !r.serial) {
    if (!g->stats) CUDA_TRY(cudaMalloc(&g->stats, kStCount * sizeof(unsigned long long)));
    P.stats = g->stats;
    g->stats_valid = true;
  }

  CheckScratch cs{counters_ptr(g), g->seen_bits, g->tile_counts, g->tile_cap, nullptr, nullptr};
  g->last_bits = r.bits;
  g->last_state = P.state;
  cudaEvent_t* ev = nullptr;
  if (r.timing) {
    if ((st = ensure_hist(g)) != MM_OK) return st;
    ev = next_hist(g, units, d_pairs || d_count);
    CUDA_TRY(cudaEventRecord(ev[0], s));
  }
  CUDA_TRY(launch_prepare(P, r.bits, prepare_grid_for(g, units), s, nullptr, 0));
  if (ev) CUDA_TRY(cudaEventRecord(ev[1], s));
  L2Window win;
  if (!r.serial) {
    if ((st = win.open(g, r, s, P.state, r.word ? g->n * 4 : packed_words(g->n, r.bits) * 4)) != MM_OK) return st;
    CUDA_TRY(launch_sweep(P, r.bits, sweep_grid_for(g, r, P.lean != 0, units), r.block, s));
    if ((st = win.close()) != MM_OK) return st;
  } else {
    CUDA_TRY(launch_serial(P, r.bits, s));
  }
  if (ev) CUDA_TRY(cudaEventRecord(ev[2], s));
  if (d_pairs || d_count) {
    uint64_t* cnt = d_count;
    CUDA_TRY(launch_compact(g->n, d_mate, d_pairs, d_pairs ? cap : 0, cnt, cs, s));
  }
  if (ev) CUDA_TRY(cudaEventRecord(ev[3], s));
  CUDA_TRY(cudaMemcpyAsync(g->h_err, err_ptr(g), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (r.nosync) return MM_OK;
  return read_err(g, s);
}

mm_status mm_skipper_to_host(mm_graph* g, const mm_options* o, uint32_t* d_mate, uint32_t* h_mate,
                             uint32_t pieces, void* cuda_stream) {
  g_err[0] = 0;
  mm_status st = check_handle(g);
  if (st != MM_OK) return st;
  if (g->local_ids) return fail(MM_ERR_UNSUPPORTED, "a MM_BATCH_LOCAL_IDS handle runs batched calls only");
  if (g->coo) return fail(MM_ERR_UNSUPPORTED, "an edge list has no rows to finish in order");
  if (g->n && (!d_mate || !h_mate)) return fail(MM_ERR_ARG, "null mate");
  if (pieces < 1 || pieces > MM_MAX_PIECES)
    return fail(MM_ERR_ARG, "pieces must be 1..%u (got %u)", MM_MAX_PIECES, pieces);
  if (o && o->unit_order == MM_ORDER_DISPERSED)
    return fail(MM_ERR_UNSUPPORTED, "the launches take units in ascending order");
  Resolved r;
  if ((st = resolve(g, o, &r)) != MM_OK) return st;
  if (r.serial || r.stats || r.timing || r.use_graph)
    return fail(MM_ERR_UNSUPPORTED, "serial, stats, timing and use_graph are not available here");
  r.disperse = false;
  if (g->n) {
    cudaPointerAttributes a{};
    CUDA_TRY(cudaPointerGetAttributes(&a, h_mate));
    if (a.type != cudaMemoryTypeHost) return fail(MM_ERR_ARG, "h_mate must be page-locked host memory");
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const uint64_t units = (g->n + g->nnz + r.grain - 1) / r.grain;
  if ((st = ensure_part(g, units)) != MM_OK) return st;
  if ((st = ensure_pieces(g)) != MM_OK) return st;
  CUDA_TRY(cudaEventSynchronize(g->pieces_done));   // a call left running on another stream
  SweepParams P = make_params(g, r, d_mate);
  g->stats_valid = false;
  g->last_bits = r.bits;
  g->last_state = P.state;
  CUDA_TRY(launch_prepare(P, r.bits, prepare_grid_for(g, units), s, nullptr, 0));
  const uint64_t K = units == 0 ? 0 : (pieces < units ? pieces : units);
  // launch i takes units [i*units/K, (i+1)*units/K); after it, every row
  // before part[2 * (i+1)*units/K] (the first row of the next unit) is done
  uint64_t* hU = g->h_split;
  uint64_t* hR = g->h_split + (MM_MAX_PIECES + 1);
  for (uint64_t i = 1; i < K; ++i)
    CUDA_TRY(cudaMemcpyAsync(hR + i, g->part + 2 * (i * units / K), sizeof(uint64_t),
                             cudaMemcpyDeviceToHost, s));
  // the split rows size the copies; this also ends the previous call's reads of hU
  CUDA_TRY(cudaStreamSynchronize(s));
  for (uint64_t i = 0; i < K; ++i) hU[i] = i * units / K;
  L2Window win;
  if ((st = win.open(g, r, s, P.state, r.word ? g->n * 4 : packed_words(g->n, r.bits) * 4)) != MM_OK) return st;
  const int grid = sweep_grid_for(g, r, P.lean != 0, units);
  uint64_t done_rows = 0;
  for (uint64_t i = 0; i < K; ++i) {
    if (i > 0)   // the unit counter starts at this launch's first unit
      CUDA_TRY(cudaMemcpyAsync(work_ptr(g), hU + i, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    SweepParams Pi = P;
    Pi.units = (i + 1) * units / K;
    CUDA_TRY(launch_sweep(Pi, r.bits, grid, r.block, s));
    const uint64_t rows = i + 1 == K ? g->n : (hR[i + 1] < g->n ? hR[i + 1] : g->n);
    if (rows > done_rows) {
      CUDA_TRY(cudaEventRecord(g->piece_ev[i], s));
      CUDA_TRY(cudaStreamWaitEvent(g->copy_stream, g->piece_ev[i], 0));
      CUDA_TRY(cudaMemcpyAsync(h_mate + done_rows, d_mate + done_rows, (rows - done_rows) * sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, g->copy_stream));
      done_rows = rows;
    }
  }
  if ((st = win.close()) != MM_OK) return st;
  if (g->n > done_rows)   // no units (a graph of isolated vertices): the prepared mate
    CUDA_TRY(cudaMemcpyAsync(h_mate + done_rows, d_mate + done_rows, (g->n - done_rows) * sizeof(uint32_t),
                             cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaEventRecord(g->piece_ev[MM_MAX_PIECES], g->copy_stream));
  CUDA_TRY(cudaStreamWaitEvent(s, g->piece_ev[MM_MAX_PIECES], 0));
  CUDA_TRY(cudaMemcpyAsync(g->h_err, err_ptr(g), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaEventRecord(g->pieces_done, s));
  if (r.nosync) return MM_OK;
  return read_err(g, s);
}

mm_status mm_sync(mm_graph* g, void* cuda_stream) {
  g_err[0] = 0;
  mm_status st = check_handle(g);
  if (st != MM_OK) return st;
  return read_err(g, static_cast<cudaStream_t>(cuda_stream));
}

mm_status mm_get_stats(mm_graph* g, mm_stats* out, void* cuda_stream) {
  if (!g || !out) return fail(MM_ERR_ARG, "null argument");
  if (!g->stats_valid) return fail(MM_ERR_ARG, "no mm_skipper call with stats = 1");
  static_assert(sizeof(mm_stats) == kStCount * sizeof(unsigned long long), "mm_stats layout");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  CUDA_TRY(cudaMemcpyAsync(out, g->stats, sizeof(mm_stats), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return MM_OK;
}

mm_status mm_state_census(mm_graph* g, uint64_t out[4], void* cuda_stream) {
  g_err[0] = 0;
  mm_status st = check_handle(g);
  if (st != MM_OK) return st;
  if (!out) return fail(MM_ERR_ARG, "null out");
  if (!g->last_state && g->n) return fail(MM_ERR_ARG, "no mm_skipper call on this handle");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  unsigned long long* d = counters_ptr(g);  // the checker's counters, free between calls
  CUDA_TRY(launch_census(g->last_state, g->n, g->last_bits ? g->last_bits : 8, d, prepare_grid(g), s));
  CUDA_TRY(cudaMemcpyAsync(g->h_counters, d, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  for (int k = 0; k < 4; ++k) out[k] = g->h_counters[k];
  return MM_OK;
}

mm_status mm_get_timing(mm_graph* g, mm_timing* out) {
  if (!g || !out) return fail(MM_ERR_ARG, "null argument");
  if (g->hist_count == 0) return fail(MM_ERR_ARG, "no timed call since the last history read");
  return read_slot(g, (uint32_t)((g->hist_count - 1) % mm_graph::kHist), out);
}

mm_status mm_timing_history(mm_graph* g, mm_timing* out, uint32_t max, uint32_t* count) {
  if (!g || !count || (max && !out)) return fail(MM_ERR_ARG, "null argument");
  const uint64_t have = g->hist_count < mm_graph::kHist ? g->hist_count : mm_graph::kHist;
  const uint32_t k = (uint32_t)(have < max ? have : max);
  for (uint32_t i = 0; i < k; ++i) {  // oldest first among the latest k calls
    const uint64_t call = g->hist_count - k + i;
    mm_status st = read_slot(g, (uint32_t)(call % mm_graph::kHist), out + i);
    if (st != MM_OK) return st;
  }
  *count = k;
  g->hist_count = 0;
  return MM_OK;
}

}  // extern "C"

namespace {

mm_status build_batch_graph(mm_graph* g, const Resolved& r, uint64_t num_graphs, bool with_pairs,
                            const SweepParams& P, uint64_t* graph_pairs) {
  BatchGraph& b = g->bg;
  if (b.exec) cudaGraphExecDestroy(b.exec);
  if (b.graph) cudaGraphDestroy(b.graph);
  b = BatchGraph{};
  CUDA_TRY(cudaGraphCreate(&b.graph, 0));
  const void *k_prepare = nullptr, *k_sweep = nullptr, *k_pairs = nullptr;
  get_batched_kernels(r.bits, r.serial, P.sym != 0, P.lean != 0, &k_prepare, &k_sweep, &k_pairs);

  SweepParams p = P;
  uint64_t* gp = graph_pairs;
  uint64_t ng = num_graphs;
  void* prep_args[] = {&p, &gp, &ng};
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void*>(k_prepare);
  kp.gridDim = dim3(prepare_grid(g));
  kp.blockDim = dim3(256);
  kp.kernelParams = prep_args;
  CUDA_TRY(cudaGraphAddKernelNode(&b.n_prepare, b.graph, nullptr, 0, &kp));

  void* sweep_args[] = {&p};
  cudaKernelNodeParams ks{};
  ks.func = const_cast<void*>(k_sweep);
  if (r.serial) {
    ks.gridDim = dim3((unsigned)((num_graphs + 127) / 128));
    ks.blockDim = dim3(128);
  } else {
    ks.gridDim = dim3(sweep_grid(g, r, P.lean != 0));
    ks.blockDim = dim3(r.block);
  }
  ks.kernelParams = sweep_args;
  CUDA_TRY(cudaGraphAddKernelNode(&b.n_sweep, b.graph, &b.n_prepare, 1, &ks));
  cudaGraphNode_t last = b.n_sweep;

  if (with_pairs) {
    const uint32_t* mate = P.mate;
    const int64_t* vb = P.vbase;
    uint64_t n = g->n;
    unsigned long long* out = reinterpret_cast<unsigned long long*>(graph_pairs);
    void* pair_args[] = {&mate, &vb, &ng, &n, &out};
    cudaKernelNodeParams kq{};
    kq.func = const_cast<void*>(k_pairs);
    kq.gridDim = dim3(prepare_grid(g));
    kq.blockDim = dim3(256);
    kq.kernelParams = pair_args;
    CUDA_TRY(cudaGraphAddKernelNode(&b.n_pairs, b.graph, &last, 1, &kq));
    last = b.n_pairs;
  }
  CUDA_TRY(cudaGraphAddMemcpyNode1D(&b.n_copy, b.graph, &last, 1, g->h_err, err_ptr(g),
                                    sizeof(uint32_t), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaGraphInstantiate(&b.exec, b.graph, 0));
  b.valid = true;
  b.status_bits = (uint32_t)r.bits;
  b.serial = r.serial;
  b.sym = r.sym;
  b.grain = r.grain;
  b.block = (uint32_t)r.block;
  b.blocks_per_sm = (uint32_t)r.blocks_per_sm;
  b.with_pairs = with_pairs;
  b.num_graphs = num_graphs;
  return MM_OK;
}

mm_status update_batch_graph(mm_graph* g, const Resolved& r, uint64_t num_graphs,
                             const SweepParams& P, uint64_t* graph_pairs) {
  BatchGraph& b = g->bg;
  const void *k_prepare = nullptr, *k_sweep = nullptr, *k_pairs = nullptr;
  get_batched_kernels(r.bits, r.serial, P.sym != 0, P.lean != 0, &k_prepare, &k_sweep, &k_pairs);
  SweepParams p = P;
  uint64_t* gp = graph_pairs;
  uint64_t ng = num_graphs;
  void* prep_args[] = {&p, &gp, &ng};
  cudaKernelNodeParams kp{};
  CUDA_TRY(cudaGraphKernelNodeGetParams(b.n_prepare, &kp));
  kp.kernelParams = prep_args;
  kp.extra = nullptr;
  CUDA_TRY(cudaGraphExecKernelNodeSetParams(b.exec, b.n_prepare, &kp));
  void* sweep_args[] = {&p};
  cudaKernelNodeParams ks{};
  CUDA_TRY(cudaGraphKernelNodeGetParams(b.n_sweep, &ks));
  ks.kernelParams = sweep_args;
  ks.extra = nullptr;
  CUDA_TRY(cudaGraphExecKernelNodeSetParams(b.exec, b.n_sweep, &ks));
  if (b.with_pairs) {
    const uint32_t* mate = P.mate;
    const int64_t* vb = P.vbase;
    uint64_t n = g->n;
    unsigned long long* out = reinterpret_cast<unsigned long long*>(graph_pairs);
    void* pair_args[] = {&mate, &vb, &ng, &n, &out};
    cudaKernelNodeParams kq{};
    CUDA_TRY(cudaGraphKernelNodeGetParams(b.n_pairs, &kq));
    kq.kernelParams = pair_args;
    kq.extra = nullptr;
    CUDA_TRY(cudaGraphExecKernelNodeSetParams(b.exec, b.n_pairs, &kq));
  }
  return MM_OK;
}

// ---- batches partitioned per member graph (batch.cu) ----

// Device tables for num_graphs graphs split into units of at least `grain`
// items: ubase / sbase / totals, unit -> graph, unit starts; and room for the
// states of every graph at a word boundary of its own.
mm_status ensure_batch_scratch(mm_graph* g, uint64_t num_graphs, uint64_t grain, int bits) {
  if (!g->btab || g->btab_graphs < num_graphs) {
    if (g->btab) cudaFree(g->btab);
    g->btab = nullptr;
    g->btab_graphs = 0;
    CUDA_TRY(cudaMalloc(&g->btab, (2 * (num_graphs + 1) + 2) * sizeof(uint64_t)));
    g->btab_graphs = num_graphs;
  }
  // sum over graphs of ceil(items_g / grain) <= (n + nnz) / grain + num_graphs
  const uint64_t units = (g->n + g->nnz) / grain + num_graphs + 1;
  if (!g->bgid || g->bunits_cap < units) {
    if (g->bgid) cudaFree(g->bgid);
    if (g->bpart) cudaFree(g->bpart);
    g->bgid = nullptr;
    g->bpart = nullptr;
    g->bunits_cap = 0;
    CUDA_TRY(cudaMalloc(&g->bgid, (units + 1) * sizeof(uint32_t)));
    CUDA_TRY(cudaMalloc(&g->bpart, 2 * (units + 1) * sizeof(int64_t)));
    g->bunits_cap = units;
  }
  if (bits != 32) {
    const uint64_t words = packed_words(g->n, bits) + (g->local_ids ? num_graphs : 0) + 4;
    if (g->state_words < words) {
      cudaFree(g->state);
      g->state = nullptr;
      g->state_words = 0;
      CUDA_TRY(cudaMalloc(&g->state, words * sizeof(uint32_t)));
      g->state_words = words;
    }
  }
  return MM_OK;
}

BatchParams batch_params(mm_graph* g, const Resolved& r, uint64_t num_graphs, const int64_t* d_vbase,
                         const int64_t* d_ebase, uint32_t* d_mate, uint64_t* d_graph_pairs) {
  BatchParams B{};
  B.P.n = g->n;
  B.P.nnz = g->nnz;
  B.P.offsets = g->offsets;
  B.P.nbrs = g->nbrs;
  B.P.mate = d_mate;
  B.P.state = r.word ? d_mate : g->state;
  B.P.work = work_ptr(g);
  B.P.err = err_ptr(g);
  B.P.spin_limit = r.spin_limit;
  B.P.disperse = r.disperse ? 1u : 0u;
  B.vbase = d_vbase;
  B.ebase = d_ebase;
  B.num_graphs = num_graphs;
  B.ubase = g->btab;
  B.sbase = g->btab + num_graphs + 1;
  B.totals = g->btab + 2 * (num_graphs + 1);
  B.gid = g->bgid;
  B.part = g->bpart;
  B.grain = r.grain;
  B.wpg = r.wpg;
  B.local = g->local_ids ? 1u : 0u;
  B.graph_pairs = d_graph_pairs;
  return B;
}

struct BatchLaunch {
  BatchKernels k;
  dim3 plan_grid, plan_block, prep_grid, prep_block, sweep_grid, sweep_block, pairs_grid, pairs_block;
};

BatchLaunch batch_launch(const mm_graph* g, const Resolved& r, uint64_t num_graphs) {
  BatchLaunch L{};
  const bool lean = r.lean && !r.serial;
  get_batch_kernels(r.bits, g->local_ids, r.serial, r.sym && !r.serial, lean, &L.k);
  L.plan_grid = dim3(1);
  L.plan_block = dim3(batch_plan_threads());
  L.prep_grid = dim3(prepare_grid(g));
  L.prep_block = dim3(256);
  if (r.serial) {
    L.sweep_grid = dim3((unsigned)((num_graphs + 127) / 128));
    L.sweep_block = dim3(128);
  } else {
    const int per_sm = r.blocks_per_sm > 0 ? r.blocks_per_sm
                                           : batch_sweep_blocks_per_sm(r.bits, g->local_ids, r.sym, lean, r.block);
    L.sweep_grid = dim3(g->num_sms * per_sm);
    L.sweep_block = dim3(r.block);
  }
  L.pairs_grid = dim3(prepare_grid(g));
  L.pairs_block = dim3(256);
  return L;
}

// A CUDA graph of the launches: plan -> prepare -> sweep -> (pairs) -> status copy.
mm_status build_batch_graph2(mm_graph* g, const Resolved& r, uint64_t num_graphs, BatchParams B) {
  BatchGraph& b = g->bg2;
  if (b.exec) cudaGraphExecDestroy(b.exec);
  if (b.graph) cudaGraphDestroy(b.graph);
  b = BatchGraph{};
  const BatchLaunch L = batch_launch(g, r, num_graphs);
  CUDA_TRY(cudaGraphCreate(&b.graph, 0));
  int states = 1;
  void* a1[] = {&B};
  void* a2[] = {&B, &states};
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void*>(L.k.plan);
  kp.gridDim = L.plan_grid;
  kp.blockDim = L.plan_block;
  kp.kernelParams = a1;
  CUDA_TRY(cudaGraphAddKernelNode(&b.n_plan, b.graph, nullptr, 0, &kp));
  kp.func = const_cast<void*>(L.k.prepare);
  kp.gridDim = L.prep_grid;
  kp.blockDim = L.prep_block;
  kp.kernelParams = a2;
  CUDA_TRY(cudaGraphAddKernelNode(&b.n_prepare, b.graph, &b.n_plan, 1, &kp));
  kp.func = const_cast<void*>(L.k.sweep);
  kp.gridDim = L.sweep_grid;
  kp.blockDim = L.sweep_block;
  kp.kernelParams = a1;
  CUDA_TRY(cudaGraphAddKernelNode(&b.n_sweep, b.graph, &b.n_prepare, 1, &kp));
  cudaGraphNode_t last = b.n_sweep;
  if (B.graph_pairs) {
    kp.func = const_cast<void*>(L.k.pairs);
    kp.gridDim = L.pairs_grid;
    kp.blockDim = L.pairs_block;
    kp.kernelParams = a1;
    CUDA_TRY(cudaGraphAddKernelNode(&b.n_pairs, b.graph, &last, 1, &kp));
    last = b.n_pairs;
  }
  CUDA_TRY(cudaGraphAddMemcpyNode1D(&b.n_copy, b.graph, &last, 1, g->h_err, err_ptr(g), sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaGraphInstantiate(&b.exec, b.graph, 0));
  b.valid = true;
  b.status_bits = (uint32_t)r.bits;
  b.serial = r.serial;
  b.sym = r.sym;
  b.grain = r.grain;
  b.wpg = r.wpg;
  b.block = (uint32_t)r.block;
  b.blocks_per_sm = (uint32_t)r.blocks_per_sm;
  b.with_pairs = B.graph_pairs != nullptr;
  b.num_graphs = num_graphs;
  return MM_OK;
}

// New arguments (buffers, tables) for the kernel nodes of the built graph.
mm_status update_batch_graph2(mm_graph* g, BatchParams B) {
  BatchGraph& b = g->bg2;
  int states = 1;
  void* a1[] = {&B};
  void* a2[] = {&B, &states};
  cudaGraphNode_t nodes[] = {b.n_plan, b.n_prepare, b.n_sweep, b.n_pairs};
  for (int i = 0; i < 4; ++i) {
    if (!nodes[i]) continue;
    cudaKernelNodeParams kp{};
    CUDA_TRY(cudaGraphKernelNodeGetParams(nodes[i], &kp));
    kp.kernelParams = i == 1 ? a2 : a1;
    kp.extra = nullptr;
    CUDA_TRY(cudaGraphExecKernelNodeSetParams(b.exec, nodes[i], &kp));
  }
  return MM_OK;
}

mm_status run_batched2(mm_graph* g, const Resolved& r, uint64_t num_graphs, const int64_t* d_vbase,
                       const int64_t* d_ebase, uint32_t* d_mate, uint64_t* d_graph_pairs, cudaStream_t s) {
  if (r.stats || r.poison)
    return fail(MM_ERR_UNSUPPORTED, "stats and poison_vertex are not available with local ids or warps_per_graph");
  if (num_graphs >= (1ull << 32)) return fail(MM_ERR_ARG, "num_graphs must stay below 2^32");
  mm_status st;
  if ((st = ensure_batch_scratch(g, num_graphs, r.grain, r.bits)) != MM_OK) return st;
  BatchParams B = batch_params(g, r, num_graphs, d_vbase, d_ebase, d_mate, d_graph_pairs);
  if (r.use_graph) {
    BatchGraph& b = g->bg2;
    const bool same = b.valid && b.status_bits == (uint32_t)r.bits && b.serial == (uint32_t)r.serial &&
                      b.sym == r.sym && b.grain == r.grain && b.wpg == r.wpg && b.block == (uint32_t)r.block &&
                      b.blocks_per_sm == (uint32_t)r.blocks_per_sm && b.with_pairs == (d_graph_pairs != nullptr) &&
                      b.num_graphs == num_graphs;
    if (!same) {
      if ((st = build_batch_graph2(g, r, num_graphs, B)) != MM_OK) return st;
    } else {
      if ((st = update_batch_graph2(g, B)) != MM_OK) return st;
    }
    CUDA_TRY(cudaGraphLaunch(b.exec, s));
    if (r.nosync) return MM_OK;
    return read_err(g, s);
  }
  const BatchLaunch L = batch_launch(g, r, num_graphs);
  cudaEvent_t* ev = nullptr;
  if (r.timing) {
    if ((st = ensure_hist(g)) != MM_OK) return st;
    ev = next_hist(g, 0, d_graph_pairs != nullptr);
    CUDA_TRY(cudaEventRecord(ev[0], s));
  }
  int states = 1;
  void* a1[] = {&B};
  void* a2[] = {&B, &states};
  CUDA_TRY(cudaLaunchKernel(L.k.plan, L.plan_grid, L.plan_block, a1, 0, s));
  CUDA_TRY(cudaLaunchKernel(L.k.prepare, L.prep_grid, L.prep_block, a2, 0, s));
  if (ev) CUDA_TRY(cudaEventRecord(ev[1], s));
  CUDA_TRY(cudaLaunchKernel(L.k.sweep, L.sweep_grid, L.sweep_block, a1, 0, s));
  if (ev) CUDA_TRY(cudaEventRecord(ev[2], s));
  if (d_graph_pairs) CUDA_TRY(cudaLaunchKernel(L.k.pairs, L.pairs_grid, L.pairs_block, a1, 0, s));
  if (ev) CUDA_TRY(cudaEventRecord(ev[3], s));
  CUDA_TRY(cudaMemcpyAsync(g->h_err, err_ptr(g), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (r.nosync) return MM_OK;
  return read_err(g, s);
}

}  // namespace

extern "C" {

mm_status mm_skipper_batched(mm_graph* g, uint64_t num_graphs, const int64_t* d_vbase,
                             const int64_t* d_ebase, const mm_options* o, uint32_t* d_mate,
                             uint64_t* d_graph_pairs, void* cuda_stream) {
  g_err[0] = 0;
  mm_status st = check_handle(g);
  if (st != MM_OK) return st;
  if (g->coo) return fail(MM_ERR_UNSUPPORTED, "batched calls take a CSR handle");
  if (num_graphs == 0) return fail(MM_ERR_ARG, "num_graphs = 0");
  if (!d_vbase || !d_ebase) return fail(MM_ERR_ARG, "null vbase / ebase");
  if (!d_mate && g->n) return fail(MM_ERR_ARG, "null mate");
  Resolved r;
  if ((st = resolve(g, o, &r)) != MM_OK) return st;
  if (r.timing && r.use_graph) return fail(MM_ERR_UNSUPPORTED, "timing with use_graph");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (g->local_ids || r.wpg)
    return run_batched2(g, r, num_graphs, d_vbase, d_ebase, d_mate, d_graph_pairs, s);
  const uint64_t units = (g->n + g->nnz + r.grain - 1) / r.grain;
  if ((st = ensure_part(g, units)) != MM_OK) return st;
  SweepParams P = make_params(g, r, d_mate);
  P.sel = 0;  // batched sweeps load ids eagerly (the graph-launched ones share one kernel)
  P.tile = 0;
  P.vbase = d_vbase;
  P.num_graphs = num_graphs;
  (void)d_ebase;  // entry ranges follow from offsets[vbase[k]]; kept in the ABI for callers

  if (r.use_graph) {
    BatchGraph& b = g->bg;
    const bool with_pairs = d_graph_pairs != nullptr;
    const bool same = b.valid && b.status_bits == (uint32_t)r.bits && b.serial == (uint32_t)r.serial &&
                      b.sym == r.sym &&
                      b.grain == r.grain && b.block == (uint32_t)r.block &&
                      b.blocks_per_sm == (uint32_t)r.blocks_per_sm && b.with_pairs == with_pairs &&
                      b.num_graphs == num_graphs && units <= g->part_units_cap;
    if (!same) {
      if ((st = build_batch_graph(g, r, num_graphs, with_pairs, P, d_graph_pairs)) != MM_OK) return st;
    } else {
      if ((st = update_batch_graph(g, r, num_graphs, P, d_graph_pairs)) != MM_OK) return st;
    }
    CUDA_TRY(cudaGraphLaunch(b.exec, s));
    if (r.nosync) return MM_OK;
    return read_err(g, s);
  }

  cudaEvent_t* ev = nullptr;
  if (r.timing) {
    if ((st = ensure_hist(g)) != MM_OK) return st;
    ev = next_hist(g, units, d_graph_pairs != nullptr);
    CUDA_TRY(cudaEventRecord(ev[0], s));
  }
  CUDA_TRY(launch_prepare(P, r.bits, prepare_grid(g), s, d_graph_pairs, d_graph_pairs ? num_graphs : 0));
  if (ev) CUDA_TRY(cudaEventRecord(ev[1], s));
  if (r.serial)
    CUDA_TRY(launch_serial_batched(P, r.bits, s));
  else
    CUDA_TRY(launch_sweep(P, r.bits, sweep_grid(g, r, P.lean != 0), r.block, s));
  if (ev) CUDA_TRY(cudaEventRecord(ev[2], s));
  if (d_graph_pairs)
    CUDA_TRY(launch_graph_pairs(d_mate, d_vbase, num_graphs, g->n, d_graph_pairs, prepare_grid(g), s));
  if (ev) CUDA_TRY(cudaEventRecord(ev[3], s));
  CUDA_TRY(cudaMemcpyAsync(g->h_err, err_ptr(g), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (r.nosync) return MM_OK;
  return read_err(g, s);
}

mm_status mm_validate(mm_graph* g, const uint32_t* d_mate, const uint32_t* d_pairs, uint64_t count,
                      mm_verdict* h_out, void* cuda_stream) {
  g_err[0] = 0;
  mm_status st = check_handle(g);
  if (st != MM_OK) return st;
  if (g->local_ids) return fail(MM_ERR_UNSUPPORTED, "a MM_BATCH_LOCAL_IDS handle is checked by mm_validate_batched");
  if (!h_out) return fail(MM_ERR_ARG, "null verdict");
  if (!d_mate && g->n) return fail(MM_ERR_ARG, "null mate");
  if (d_pairs && count && !g->seen_bits)
    CUDA_TRY(cudaMalloc(&g->seen_bits, ((g->n + 31) / 32 + 1) * sizeof(uint32_t)));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (g->coo) {
    if (!g->found) CUDA_TRY(cudaMalloc(&g->found, g->n + 16));
    CheckScratch cs{counters_ptr(g), g->seen_bits, g->tile_counts, g->tile_cap, g->found, nullptr};
    CUDA_TRY(launch_validate_coo(g->n, g->nnz, g->src, g->dst, d_mate, d_pairs, d_pairs ? count : 0, cs,
                                 prepare_grid(g), s));
  } else {
    if (!g->check_part)
      CUDA_TRY(cudaMalloc(&g->check_part, ((g->n + g->nnz) / kCheckGrain + 2) * 2 * sizeof(int64_t)));
    CheckScratch cs{counters_ptr(g), g->seen_bits, g->tile_counts, g->tile_cap, nullptr, g->check_part};
    CUDA_TRY(launch_validate(g->n, g->nnz, g->offsets, g->nbrs, d_mate, d_pairs, d_pairs ? count : 0, cs,
                             prepare_grid(g), s));
  }
  CUDA_TRY(cudaMemcpyAsync(g->h_counters, counters_ptr(g), 9 * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const unsigned long long* c = g->h_counters;
  mm_verdict v{};
  v.n_matched = c[0];
  v.n_pairs = c[1];
  v.n_bad_range = c[2];
  v.n_asym = c[3];
  v.n_nonedge = c[4];
  v.n_uncovered = c[5];
  v.n_pairs_bad = c[6];
  v.first_bad_vertex = c[7];
  v.first_uncovered = c[8];
  if (v.n_bad_range) v.flags |= MM_V_RANGE;
  if (v.n_asym) v.flags |= MM_V_ASYM;
  if (v.n_nonedge) v.flags |= MM_V_NONEDGE;
  if (v.n_uncovered) v.flags |= MM_V_UNCOVERED;
  if (d_pairs && (v.n_pairs_bad || count != v.n_pairs)) v.flags |= MM_V_PAIRS;
  *h_out = v;
  return MM_OK;
}

mm_status mm_validate_batched(mm_graph* g, uint64_t num_graphs, const int64_t* d_vbase,
                              const int64_t* d_ebase, const uint32_t* d_mate, mm_verdict* h_out,
                              void* cuda_stream) {
  g_err[0] = 0;
  mm_status st = check_handle(g);
  if (st != MM_OK) return st;
  if (g->coo) return fail(MM_ERR_UNSUPPORTED, "batched calls take a CSR handle");
  if (!h_out) return fail(MM_ERR_ARG, "null verdict");
  if (num_graphs == 0 || num_graphs >= (1ull << 32)) return fail(MM_ERR_ARG, "num_graphs must be in [1, 2^32)");
  if (!d_vbase || !d_ebase) return fail(MM_ERR_ARG, "null vbase / ebase");
  if (!d_mate && g->n) return fail(MM_ERR_ARG, "null mate");
  if ((st = ensure_batch_scratch(g, num_graphs, kCheckGrain, 32)) != MM_OK) return st;
  Resolved r{};
  r.grain = (uint32_t)kCheckGrain;
  r.bits = 32;
  r.word = true;
  const BatchParams B = batch_params(g, r, num_graphs, d_vbase, d_ebase, const_cast<uint32_t*>(d_mate), nullptr);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  CUDA_TRY(launch_validate_batch(B, counters_ptr(g), prepare_grid(g), s));
  CUDA_TRY(cudaMemcpyAsync(g->h_counters, counters_ptr(g), 9 * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const unsigned long long* c = g->h_counters;
  mm_verdict v{};
  v.n_matched = c[0];
  v.n_pairs = c[1];
  v.n_bad_range = c[2];
  v.n_asym = c[3];
  v.n_nonedge = c[4];
  v.n_uncovered = c[5];
  v.n_pairs_bad = c[6];
  v.first_bad_vertex = c[7];
  v.first_uncovered = c[8];
  if (v.n_bad_range) v.flags |= MM_V_RANGE;
  if (v.n_asym) v.flags |= MM_V_ASYM;
  if (v.n_nonedge) v.flags |= MM_V_NONEDGE;
  if (v.n_uncovered) v.flags |= MM_V_UNCOVERED;
  *h_out = v;
  return MM_OK;
}

mm_status mm_autotune(mm_graph* g, uint32_t* d_mate_scratch, mm_options* o, void* cuda_stream) {
  g_err[0] = 0;
  mm_status st = check_handle(g);
  if (st != MM_OK) return st;
  if (!o || (!d_mate_scratch && g->n)) return fail(MM_ERR_ARG, "null options or scratch");
  if (g->local_ids) return fail(MM_ERR_UNSUPPORTED, "a MM_BATCH_LOCAL_IDS handle is tuned by mm_autotune_batched");
  static const uint32_t grains[] = {2048, 8192};
  static const uint32_t bits[] = {2, 8, 32};
  const uint32_t bt = 512;
  float best = 1e30f;
  mm_options best_o = *o;
  for (uint32_t gr : grains)
    for (uint32_t sb : bits)
      for (int lean = 0; lean < 2; ++lean)
        for (uint32_t ord : {MM_ORDER_ASCENDING, MM_ORDER_DISPERSED}) {
          if (g->coo && (lean || ord == MM_ORDER_DISPERSED)) continue;  // edge lists: one instance, one order
          const uint32_t bps = g->coo ? 0u : (uint32_t)sweep_blocks_per_sm((int)sb, (int)bt, lean != 0);
          mm_options c = *o;
          c.grain = gr;
          c.status_bits = sb;
          c.block_threads = bt;
          c.blocks_per_sm = bps;
          c.unit_order = ord;
          c.serial = 0;
          c.nosync = 0;
          c.stats = 0;
          c.timing = 1;
          // one untimed run, then timed runs; dropped once 1.5x slower than the best run so far
          float total = 0;
          int reps = 0;
          bool dropped = false;
          for (int rep = 0; rep < 4; ++rep) {
            if ((st = mm_skipper(g, &c, d_mate_scratch, nullptr, 0, nullptr, cuda_stream)) != MM_OK) return st;
            mm_timing t;
            if ((st = mm_get_timing(g, &t)) != MM_OK) return st;
            if (rep == 0) continue;
            total += t.total_ms;
            ++reps;
            if (rep == 1 && best < 1e30f && t.total_ms > 1.5f * (best / 3.0f)) {
              dropped = true;
              break;
            }
          }
          if (dropped || reps != 3 || total >= best) continue;
          mm_verdict v;
          if ((st = mm_validate(g, d_mate_scratch, nullptr, 0, &v, cuda_stream)) != MM_OK) return st;
          if (v.flags) return fail(MM_ERR_CUDA, "autotune candidate gave an invalid matching (flags 0x%x)", v.flags);
          best = total;
          best_o = *o;
          best_o.grain = gr;
          best_o.status_bits = sb;
          best_o.block_threads = bt;
          best_o.blocks_per_sm = bps;
          best_o.unit_order = ord;
        }
  *o = best_o;
  return MM_OK;
}

mm_status mm_autotune_batched(mm_graph* g, uint64_t num_graphs, const int64_t* d_vbase,
                              const int64_t* d_ebase, uint32_t* d_mate_scratch, mm_options* o,
                              void* cuda_stream) {
  g_err[0] = 0;
  mm_status st = check_handle(g);
  if (st != MM_OK) return st;
  if (!o || !d_mate_scratch) return fail(MM_ERR_ARG, "null options or scratch");
  if (g->coo) return fail(MM_ERR_UNSUPPORTED, "batched calls take a CSR handle");
  static const uint32_t grains[] = {1024, 2048, 4096, 8192};
  static const uint32_t bits[] = {2, 8, 32};
  static const uint32_t wpgs[] = {0, 4, 16};
  const uint32_t bt = 512;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  float best = 1e30f;
  mm_options best_o = *o;
  for (uint32_t gr : grains)
    for (uint32_t sb : bits)
      for (int lean = 0; lean < 2; ++lean)
        for (uint32_t ord : {MM_ORDER_ASCENDING, MM_ORDER_DISPERSED})
        for (uint32_t wg : wpgs) {
        // occupancy: the blocks per SM of the 40- or the 32-register instance
        const uint32_t bps = (uint32_t)sweep_blocks_per_sm((int)sb, (int)bt, lean != 0);
        mm_options c = *o;
        c.grain = gr;
        c.status_bits = sb;
        c.block_threads = bt;
        c.blocks_per_sm = bps;
        c.unit_order = ord;
        c.warps_per_graph = wg;
        c.serial = 0;
        c.use_graph = 0;
        c.nosync = 0;
        c.timing = 1;
        // one untimed run, one timed run; a candidate already 1.5x slower than
        // the best per run is dropped, the others get two more timed runs
        float total = 0;
        int reps = 0;
        bool dropped = false;
        for (int rep = 0; rep < 4; ++rep) {
          if ((st = mm_skipper_batched(g, num_graphs, d_vbase, d_ebase, &c, d_mate_scratch, nullptr, s)) != MM_OK)
            return st;
          mm_timing t;
          if ((st = mm_get_timing(g, &t)) != MM_OK) return st;
          if (rep == 0) continue;
          total += t.total_ms;
          ++reps;
          if (rep == 1 && best < 1e30f && t.total_ms > 1.5f * (best / 3.0f)) {
            dropped = true;
            break;
          }
        }
        if (dropped || reps != 3 || total >= best) continue;
        mm_verdict v;
        if ((st = mm_validate_batched(g, num_graphs, d_vbase, d_ebase, d_mate_scratch, &v, s)) != MM_OK) return st;
        if (v.flags) return fail(MM_ERR_CUDA, "autotune candidate gave an invalid matching (flags 0x%x)", v.flags);
        best = total;
        best_o = *o;
        best_o.grain = gr;
        best_o.status_bits = sb;
        best_o.block_threads = bt;
        best_o.blocks_per_sm = bps;
        best_o.unit_order = ord;
        best_o.warps_per_graph = wg;
        }
  *o = best_o;
  return MM_OK;
}

mm_status mm_destroy(mm_graph* g) {
  if (!g) return MM_OK;
  if (g->bg.exec) cudaGraphExecDestroy(g->bg.exec);
  if (g->bg.graph) cudaGraphDestroy(g->bg.graph);
  if (g->bg2.exec) cudaGraphExecDestroy(g->bg2.exec);
  if (g->bg2.graph) cudaGraphDestroy(g->bg2.graph);
  if (g->btab) cudaFree(g->btab);
  if (g->bgid) cudaFree(g->bgid);
  if (g->bpart) cudaFree(g->bpart);
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  for (auto& set : g->hist)
    for (auto& e : set)
      if (e) cudaEventDestroy(e);
  if (g->state) cudaFree(g->state);
  if (g->part) cudaFree(g->part);
  if (g->ctrl) cudaFree(g->ctrl);
  if (g->seen_bits) cudaFree(g->seen_bits);
  if (g->found) cudaFree(g->found);
  if (g->stats) cudaFree(g->stats);
  if (g->check_part) cudaFree(g->check_part);
  if (g->tile_counts) cudaFree(g->tile_counts);
  if (g->h_err) cudaFreeHost(g->h_err);
  if (g->h_counters) cudaFreeHost(g->h_counters);
  for (auto& e : g->piece_ev)
    if (e) cudaEventDestroy(e);
  if (g->pieces_done) cudaEventDestroy(g->pieces_done);
  if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
  if (g->h_split) cudaFreeHost(g->h_split);
  delete g;
  return MM_OK;
}

}  // extern "C"
