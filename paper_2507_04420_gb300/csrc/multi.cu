// multi.cu -- Skipper over many independent graphs in one persistent launch,
// each graph in its own device buffers (mm_skipper_multi), and the exact
// checker over all of them at once (mm_validate_multi).
//
// Graphs are described by a table of (n, nnz, offsets, nbrs, mate) entries
// copied to the device per call; nothing is repacked.  Every graph is split
// into merge-path units of `grain` rows + entries (as in the single-graph
// sweep, Section IV-C's equal-edge blocks), the units of all graphs are
// numbered consecutively, and persistent warps take them from one counter, so
// large and small graphs share the GPU in a single launch.  The walk of a unit
// is the single-graph walk (walk.cuh) on a view of its graph.
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>
#include <cuda_runtime.h>

#include "internal.h"
#include "skipper.h"
#include "walk.cuh"
#include "checkwalk.cuh"

using namespace skp;

namespace skp {
namespace {

struct MultiParams {
  uint64_t num_graphs;
  const mm_graph_desc* desc;  // [G]
  const uint64_t* ubase;      // [G+1] first unit of each graph
  const uint64_t* vbase;      // [G+1] first vertex of each graph (for the init pass)
  const uint64_t* sbase;      // [G+1] first packed state word of each graph
  uint32_t* state_pool;       // packed state words of all graphs (2- or 8-bit layouts)
  int64_t* part;              // (row, entry) per unit
  uint32_t* gid;              // graph of each unit
  uint64_t units;
  uint64_t grain;
  unsigned long long* work;
  uint32_t* err;
  uint64_t spin_limit;
  unsigned long long* counters;  // checker: 9 per graph
};

// last g with base[g] <= x, base[0] = 0, base ascending, g < G
__device__ __forceinline__ uint64_t find_graph(const uint64_t* base, uint64_t G, uint64_t x) {
  uint64_t lo = 0, hi = G;
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(base + mid) <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ SweepParams view(const MultiParams& M, uint64_t g, bool word) {
  const mm_graph_desc d = M.desc[g];
  SweepParams P{};
  P.n = d.n;
  P.nnz = d.nnz;
  P.offsets = d.offsets;
  P.nbrs = d.nbrs;
  P.mate = d.mate;
  P.state = word ? d.mate : M.state_pool + M.sbase[g];
  P.err = M.err;
  P.spin_limit = M.spin_limit;
  return P;
}

template <bool kWord>
__global__ void multi_prepare_kernel(MultiParams M) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t G = M.num_graphs;
  // every vertex ACC (Algorithm 1 lines 3-4), mate unmatched: 16 vertices a thread
  const uint64_t V = M.vbase[G];
  for (uint64_t c = tid; c * 16 < V; c += nthreads) {
    const uint64_t v0 = c * 16;
    uint64_t g = find_graph(M.vbase, G, v0);
    for (uint64_t v = v0; v < v0 + 16 && v < V; ++v) {
      while (v >= M.vbase[g + 1]) ++g;
      M.desc[g].mate[v - M.vbase[g]] = kNone;  // = the word state ACC
    }
  }
  if (!kWord)
    for (uint64_t i = tid; i < M.sbase[G]; i += nthreads) M.state_pool[i] = 0u;
  // merge-path units of every graph
  for (uint64_t u = tid; u < M.units; u += nthreads) {
    const uint64_t g = find_graph(M.ubase, G, u);
    const mm_graph_desc d = M.desc[g];
    const int64_t total = (int64_t)(d.n + d.nnz);
    int64_t diag = (int64_t)((u - M.ubase[g]) * M.grain);
    if (diag > total) diag = total;
    const int64_t rows = merge_path_rows(d.offsets, (int64_t)d.n, (int64_t)d.nnz, diag);
    M.part[2 * u] = rows;
    M.part[2 * u + 1] = diag - rows;
    M.gid[u] = (uint32_t)g;
  }
  if (tid == 0) {
    *M.work = 0ull;
    *M.err = 0u;
  }
}

template <class S, bool kWord, bool kSel = false>
__global__ void __launch_bounds__(512, 3) multi_sweep_kernel(MultiParams M) {
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t pol = policy_evict_first();
  for (;;) {
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(M.work, 1ull);
    w = __shfl_sync(kFull, w, 0);
    if (w >= M.units) return;
    const uint32_t g = M.gid[w];
    const SweepParams P = view(M, g, kWord);
    const int64_t row0 = M.part[2 * w];
    const int64_t e_begin = M.part[2 * w + 1];
    const int64_t e_end = (w + 1 < M.units && M.gid[w + 1] == g) ? M.part[2 * w + 3] : (int64_t)P.nnz;
    if (e_begin < e_end) sweep_unit<S, false, false, kSel>(S(P), P, row0, e_begin, e_end, lane, pol);
    if ((w & 15) == 0) {
      uint32_t e = 0;
      if (lane == 0) e = ld_relaxed(M.err);
      if (__shfl_sync(kFull, e, 0) & kErrTimeout) return;
    }
  }
}

template <class S, bool kWord>
__global__ void multi_serial_kernel(MultiParams M) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= M.num_graphs) return;
  const SweepParams P = view(M, g, kWord);
  serial_rows(S(P), P, 0, P.n);
}

enum { C_MATCHED = 0, C_PAIRS, C_RANGE, C_ASYM, C_NONEDGE, C_UNCOVERED, C_PAIRS_BAD, C_FIRST_BAD,
       C_FIRST_UNCOVERED, C_N };

__global__ void multi_counters_init_kernel(unsigned long long* c, uint64_t G) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G * C_N;
       i += (uint64_t)gridDim.x * blockDim.x)
    c[i] = (i % C_N) >= C_FIRST_BAD ? ~0ull : 0ull;
}

__device__ __forceinline__ void group_add(unsigned long long* c, unsigned peers, uint32_t v) {
  const uint32_t s = __reduce_add_sync(peers, v);
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1 && s) atomicAdd(c, (unsigned long long)s);
}

__global__ void multi_partition_kernel(MultiParams M) {
  const uint64_t G = M.num_graphs;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < M.units;
       u += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t g = find_graph(M.ubase, G, u);
    const mm_graph_desc d = M.desc[g];
    const int64_t total = (int64_t)(d.n + d.nnz);
    int64_t diag = (int64_t)((u - M.ubase[g]) * M.grain);
    if (diag > total) diag = total;
    const int64_t rows = merge_path_rows(d.offsets, (int64_t)d.n, (int64_t)d.nnz, diag);
    M.part[2 * u] = rows;
    M.part[2 * u + 1] = diag - rows;
    M.gid[u] = (uint32_t)g;
  }
}

// the checker's edge pass (checkwalk.cuh) over the units of every graph
__global__ void multi_validate_edges_kernel(MultiParams M) {
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t u = warp; u < M.units; u += nwarps) {
    const uint32_t g = M.gid[u];
    const mm_graph_desc d = M.desc[g];
    const int64_t e0 = M.part[2 * u + 1];
    const int64_t e1 = (u + 1 < M.units && M.gid[u + 1] == g) ? M.part[2 * u + 3] : (int64_t)d.nnz;
    if (e0 >= e1) continue;
    unsigned long long unc = 0, first = ~0ull;
    check_unit(d.offsets, d.nbrs, d.n, d.nnz, d.mate, M.part[2 * u], e0, e1, lane, unc, first);
    unc = warp_sum64(unc);
    first = warp_min64(first);
    if (lane == 0) {
      unsigned long long* c = M.counters + (uint64_t)g * C_N;
      if (unc) atomicAdd(c + C_UNCOVERED, unc);
      if (first != ~0ull) atomicMin(c + C_FIRST_UNCOVERED, first);
    }
  }
}

// the checker's existence pass (checkwalk.cuh) over every vertex of every
// graph: one warp per 32 consecutive vertices of the whole batch; the pairs
// whose named edge is missing are counted in their graph's counters
__global__ void multi_validate_exist_kernel(MultiParams M) {
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t G = M.num_graphs;
  const uint64_t V = M.vbase[G];
  for (uint64_t w0 = warp * 32; w0 < V; w0 += nwarps * 32) {
    const uint64_t gv = w0 + lane;
    uint64_t g = 0;
    uint32_t v = 0, m = kNone;
    bool valid = false, sym = false;
    if (gv < V) {
      g = find_graph(M.vbase, G, gv);
      const mm_graph_desc d = M.desc[g];
      v = (uint32_t)(gv - M.vbase[g]);
      m = d.mate[v];
      valid = m != kNone && m < d.n && m != v;
      sym = valid && d.mate[m] == v;
    }
    unsigned todo = __ballot_sync(kFull, valid && !(sym && m < v));
    while (todo) {
      const int j = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint64_t gj = __shfl_sync(kFull, g, j);
      const uint32_t vj = __shfl_sync(kFull, v, j), mj = __shfl_sync(kFull, m, j);
      const bool sj = __shfl_sync(kFull, sym ? 1u : 0u, j) != 0u;
      const mm_graph_desc d = M.desc[gj];
      const int64_t dv = d.offsets[vj + 1] - d.offsets[vj];
      const int64_t dm = d.offsets[mj + 1] - d.offsets[mj];
      const bool v_first = dv <= dm;  // the shorter row first
      bool hit = warp_row_has(d.offsets, d.nbrs, v_first ? vj : mj, v_first ? mj : vj, lane);
      if (!hit) hit = warp_row_has(d.offsets, d.nbrs, v_first ? mj : vj, v_first ? vj : mj, lane);
      if (!hit && lane == 0) {
        unsigned long long* c = M.counters + gj * C_N;
        atomicAdd(c + C_NONEDGE, sj ? 2ull : 1ull);
        atomicMin(c + C_FIRST_BAD, (unsigned long long)vj);
      }
    }
  }
}

// the checker's vertex pass on every vertex of every graph (range, symmetry,
// pairs), counters kept per graph
__global__ void multi_validate_kernel(MultiParams M) {
  const uint64_t G = M.num_graphs;
  const uint64_t V = M.vbase[G];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x; v0 < V; v0 += stride) {
    const uint64_t gv = v0 + threadIdx.x;
    uint64_t g = ~0ull;
    uint32_t matched = 0, pair = 0, range = 0, asym = 0;
    uint64_t first_bad = ~0ull;
    if (gv < V) {
      g = find_graph(M.vbase, G, gv);
      const mm_graph_desc d = M.desc[g];
      const uint64_t v = gv - M.vbase[g];
      const uint64_t n = d.n;
      const uint32_t m = d.mate[v];
      if (m != kNone) {
        if (m >= n || m == v) {
          range = 1;
          first_bad = v;
        } else {
          matched = 1;
          if (d.mate[m] != (uint32_t)v) {
            asym = 1;
            first_bad = v;
          } else if (v < m) {
            pair = 1;
          }
        }
      }
    }
    const unsigned active = __ballot_sync(kFull, gv < V);
    if (gv < V) {
      const unsigned peers = __match_any_sync(active, g);
      unsigned long long* c = M.counters + g * C_N;
      group_add(c + C_MATCHED, peers, matched);
      group_add(c + C_PAIRS, peers, pair);
      group_add(c + C_RANGE, peers, range);
      group_add(c + C_ASYM, peers, asym);
      if (first_bad != ~0ull) atomicMin(c + C_FIRST_BAD, (unsigned long long)first_bad);
    }
  }
}

// Grow a device buffer to at least `want` elements, ordered on the call's
// stream (cudaFreeAsync / cudaMallocAsync), so growing never waits for the
// whole device; capacity doubles so growth is rare.
template <class T>
cudaError_t grow(T** p, uint64_t* cap, uint64_t want, cudaStream_t s) {
  if (*p && *cap >= want) return cudaSuccess;
  uint64_t n = *cap ? *cap : 64;
  while (n < want) n *= 2;
  if (*p) {
    cudaError_t e = cudaFreeAsync(*p, s);
    if (e != cudaSuccess) return e;
  }
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), n * sizeof(T), s);
  if (e == cudaSuccess) *cap = n;
  return e;
}

thread_local char g_msg[512] = "";

mm_status mfail(mm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
  set_error_message("%s", g_msg);
  return st;
}

#define MTRY(expr)                                                                             \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return mfail(e_ == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA, "%s: %s", #expr, \
                   cudaGetErrorString(e_));                                                    \
  } while (0)

}  // namespace
}  // namespace skp

// Device tables of one call ([desc G | ubase G+1 | vbase G+1 | sbase G+1]),
// their pinned staging copy and the partition built on them.  The sweep and
// the checker have one set each, so a checker enqueued right behind a sweep
// never waits for the sweep's staging copy.
struct TableSet {
  unsigned char* tables = nullptr;
  uint64_t tables_cap = 0;
  unsigned char* staging = nullptr;    // pinned host copy of the tables
  uint64_t staging_cap = 0;
  cudaEvent_t staging_free = nullptr;  // the last copy out of `staging` has finished
  bool staging_pending = false;
  int64_t* part = nullptr;
  uint64_t part_cap = 0;
  uint32_t* gid = nullptr;
  uint64_t gid_cap = 0;
};

struct mm_multi {
  int device = 0;
  int num_sms = 0;
  TableSet sweep, check;
  uint32_t* pool = nullptr;
  uint64_t pool_cap = 0;
  unsigned long long* counters = nullptr;
  uint64_t counters_cap = 0;
  unsigned long long* ctrl = nullptr;  // [0] work, [1] err
  uint32_t* h_err = nullptr;           // pinned
  unsigned long long* h_counters = nullptr;
  uint64_t h_counters_cap = 0;
  uint64_t checked_graphs = 0;         // graphs of the last enqueued check
};

namespace skp {
namespace {

struct Layout {
  uint64_t units = 0;
  uint64_t bytes = 0;
  uint64_t off_ubase = 0, off_vbase = 0, off_sbase = 0;
  uint64_t total_vertices = 0, total_words = 0;
};

mm_status stage_tables(TableSet* m, uint64_t G, const mm_graph_desc* h, uint64_t grain, int bits,
                       cudaStream_t s, Layout* L) {
  L->off_ubase = G * sizeof(mm_graph_desc);
  L->off_vbase = L->off_ubase + (G + 1) * 8;
  L->off_sbase = L->off_vbase + (G + 1) * 8;
  L->bytes = L->off_sbase + (G + 1) * 8;
  if (m->staging_pending) {  // the previous call may still be copying out of the staging buffer
    MTRY(cudaEventSynchronize(m->staging_free));
    m->staging_pending = false;
  }
  if (m->staging_cap < L->bytes) {
    uint64_t cap = m->staging_cap ? m->staging_cap : 4096;   // doubling from the old size
    while (cap < L->bytes) cap *= 2;
    if (m->staging) cudaFreeHost(m->staging);
    m->staging = nullptr;
    m->staging_cap = 0;
    MTRY(cudaMallocHost(&m->staging, cap));
    m->staging_cap = cap;
  }
  MTRY(grow(&m->tables, &m->tables_cap, L->bytes, s));
  memcpy(m->staging, h, G * sizeof(mm_graph_desc));
  uint64_t* ub = reinterpret_cast<uint64_t*>(m->staging + L->off_ubase);
  uint64_t* vb = reinterpret_cast<uint64_t*>(m->staging + L->off_vbase);
  uint64_t* sb = reinterpret_cast<uint64_t*>(m->staging + L->off_sbase);
  ub[0] = vb[0] = sb[0] = 0;
  for (uint64_t g = 0; g < G; ++g) {
    ub[g + 1] = ub[g] + (h[g].n + h[g].nnz + grain - 1) / grain;
    vb[g + 1] = vb[g] + h[g].n;
    sb[g + 1] = sb[g] + (bits == 32 ? 0 : packed_words(h[g].n, bits) + 1);
  }
  L->units = ub[G];
  L->total_vertices = vb[G];
  L->total_words = sb[G];
  MTRY(cudaMemcpyAsync(m->tables, m->staging, L->bytes, cudaMemcpyHostToDevice, s));
  MTRY(cudaEventRecord(m->staging_free, s));
  m->staging_pending = true;
  return MM_OK;
}

MultiParams params(mm_multi* m, const TableSet& t, uint64_t G, const Layout& L, uint64_t grain,
                   uint64_t spin) {
  MultiParams M{};
  M.num_graphs = G;
  M.desc = reinterpret_cast<const mm_graph_desc*>(t.tables);
  M.ubase = reinterpret_cast<const uint64_t*>(t.tables + L.off_ubase);
  M.vbase = reinterpret_cast<const uint64_t*>(t.tables + L.off_vbase);
  M.sbase = reinterpret_cast<const uint64_t*>(t.tables + L.off_sbase);
  M.state_pool = m->pool;
  M.part = t.part;
  M.gid = t.gid;
  M.units = L.units;
  M.grain = grain;
  M.work = m->ctrl;
  M.err = reinterpret_cast<uint32_t*>(m->ctrl + 1);
  M.spin_limit = spin;
  M.counters = m->counters;
  return M;
}

mm_status check_descs(uint64_t G, const mm_graph_desc* h) {
  for (uint64_t g = 0; g < G; ++g) {
    const mm_graph_desc& d = h[g];
    if (d.n > MM_MAX_VERTICES) return mfail(MM_ERR_ARG, "graph %llu: n too large", (unsigned long long)g);
    if (!d.offsets || (d.nnz && !d.nbrs) || (d.n && !d.mate))
      return mfail(MM_ERR_ARG, "graph %llu: null array", (unsigned long long)g);
    if (d.nnz && (reinterpret_cast<uintptr_t>(d.nbrs) & 15u))
      return mfail(MM_ERR_ARG, "graph %llu: nbrs must be 16-byte aligned", (unsigned long long)g);
  }
  return MM_OK;
}

}  // namespace
}  // namespace skp

extern "C" {

mm_status mm_multi_create(mm_multi** out) {
  if (!out) return mfail(MM_ERR_ARG, "null out");
  *out = nullptr;
  mm_multi* m = new (std::nothrow) mm_multi();
  if (!m) return mfail(MM_ERR_OOM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&m->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
  if (e == cudaSuccess) e = cudaMalloc(&m->ctrl, 16 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMallocHost(&m->h_err, 64);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->sweep.staging_free, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->check.staging_free, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    mm_multi_destroy(m);
    return mfail(MM_ERR_CUDA, "mm_multi_create: %s", cudaGetErrorString(e));
  }
  *m->h_err = 0;
  *out = m;
  return MM_OK;
}

mm_status mm_skipper_multi(mm_multi* m, uint64_t num_graphs, const mm_graph_desc* h_descs,
                           const mm_options* o, void* cuda_stream) {
  if (!m) return mfail(MM_ERR_ARG, "null handle");
  if (!num_graphs) return MM_OK;
  if (!h_descs) return mfail(MM_ERR_ARG, "null descriptors");
  mm_status st = check_descs(num_graphs, h_descs);
  if (st != MM_OK) return st;
  mm_options d;
  mm_default_options(&d);
  if (!o) o = &d;
  const uint32_t bits = o->status_bits ? o->status_bits : 8u;
  if (bits != 2 && bits != 8 && bits != 32) return mfail(MM_ERR_ARG, "status_bits must be 2, 8 or 32");
  const bool word = bits == 32;
  const uint64_t grain = o->grain ? o->grain : 2048;
  if (grain % 128 || grain > (1u << 24)) return mfail(MM_ERR_ARG, "bad grain");
  const int block = o->block_threads ? (int)o->block_threads : 512;
  if (block < 32 || block > 512 || block % 32) return mfail(MM_ERR_ARG, "bad block_threads");
  if (o->id_loads > MM_ID_LOADS_SELECTIVE) return mfail(MM_ERR_ARG, "id_loads must be 0, 1 or 2");
  const bool sel = o->id_loads == MM_ID_LOADS_SELECTIVE;   // automatic: eager
  if (o->timing || o->use_graph || o->poison_vertex || o->l2_persist)
    return mfail(MM_ERR_UNSUPPORTED, "timing, use_graph, poison_vertex and l2_persist are not "
                                     "available in multi-graph calls");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  Layout L;
  if ((st = stage_tables(&m->sweep, num_graphs, h_descs, grain, (int)bits, s, &L)) != MM_OK) return st;
  MTRY(grow(&m->sweep.part, &m->sweep.part_cap, 2 * (L.units + 1), s));
  MTRY(grow(&m->sweep.gid, &m->sweep.gid_cap, L.units + 1, s));
  if (!word) MTRY(grow(&m->pool, &m->pool_cap, L.total_words + 1, s));
  const MultiParams M = params(m, m->sweep, num_graphs, L, grain, o->spin_limit ? o->spin_limit : (1ull << 20));

  const int prep_grid = m->num_sms * 8;
  if (word) multi_prepare_kernel<true><<<prep_grid, 256, 0, s>>>(M);
  else multi_prepare_kernel<false><<<prep_grid, 256, 0, s>>>(M);
  MTRY(cudaGetLastError());
  if (o->serial) {
    const unsigned grid = (unsigned)((num_graphs + 127) / 128);
    if (bits == 32) multi_serial_kernel<WordState, true><<<grid, 128, 0, s>>>(M);
    else if (bits == 2) multi_serial_kernel<TwoBitState, false><<<grid, 128, 0, s>>>(M);
    else multi_serial_kernel<ByteState, false><<<grid, 128, 0, s>>>(M);
  } else if (L.units) {
    int per_sm = (int)o->blocks_per_sm;
    if (per_sm <= 0) {
      cudaError_t e = bits == 32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, multi_sweep_kernel<WordState, true>, block, 0)
                    : bits == 2  ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, multi_sweep_kernel<TwoBitState, false>, block, 0)
                                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, multi_sweep_kernel<ByteState, false>, block, 0);
      if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    }
    const int grid = m->num_sms * per_sm;
    if (sel) {
      if (bits == 32) multi_sweep_kernel<WordState, true, true><<<grid, block, 0, s>>>(M);
      else if (bits == 2) multi_sweep_kernel<TwoBitState, false, true><<<grid, block, 0, s>>>(M);
      else multi_sweep_kernel<ByteState, false, true><<<grid, block, 0, s>>>(M);
    } else {
      if (bits == 32) multi_sweep_kernel<WordState, true><<<grid, block, 0, s>>>(M);
      else if (bits == 2) multi_sweep_kernel<TwoBitState, false><<<grid, block, 0, s>>>(M);
      else multi_sweep_kernel<ByteState, false><<<grid, block, 0, s>>>(M);
    }
  }
  MTRY(cudaGetLastError());
  MTRY(cudaMemcpyAsync(m->h_err, M.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (o->nosync) return MM_OK;
  return mm_multi_sync(m, cuda_stream);
}

mm_status mm_multi_sync(mm_multi* m, void* cuda_stream) {
  if (!m) return mfail(MM_ERR_ARG, "null handle");
  MTRY(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)));
  const uint32_t e = *m->h_err;
  if (e & kErrTimeout) return mfail(MM_ERR_TIMEOUT, "a wait on a reserved vertex ran past spin_limit");
  if (e & kErrBadId) return mfail(MM_ERR_BAD_GRAPH, "a neighbour id >= n was met");
  return MM_OK;
}

mm_status mm_validate_multi_async(mm_multi* m, uint64_t num_graphs, const mm_graph_desc* h_descs,
                                  void* cuda_stream) {
  if (!m) return mfail(MM_ERR_ARG, "null handle");
  m->checked_graphs = 0;
  if (!num_graphs) return MM_OK;
  if (!h_descs) return mfail(MM_ERR_ARG, "null descriptors");
  mm_status st = check_descs(num_graphs, h_descs);
  if (st != MM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  Layout L;
  if ((st = stage_tables(&m->check, num_graphs, h_descs, kCheckGrain, 32, s, &L)) != MM_OK) return st;
  MTRY(grow(&m->counters, &m->counters_cap, num_graphs * C_N, s));
  MTRY(grow(&m->check.part, &m->check.part_cap, 2 * (L.units + 1), s));
  MTRY(grow(&m->check.gid, &m->check.gid_cap, L.units + 1, s));
  if (m->h_counters_cap < num_graphs * C_N) {
    // the previous check's counters may still be on their way into the old buffer
    MTRY(cudaStreamSynchronize(s));
    if (m->h_counters) cudaFreeHost(m->h_counters);
    m->h_counters = nullptr;
    uint64_t cap = m->h_counters_cap ? m->h_counters_cap : 64 * C_N;
    while (cap < num_graphs * C_N) cap *= 2;
    m->h_counters_cap = 0;
    MTRY(cudaMallocHost(&m->h_counters, cap * sizeof(unsigned long long)));
    m->h_counters_cap = cap;
  }
  const MultiParams M = params(m, m->check, num_graphs, L, kCheckGrain, 1);
  const int grid = m->num_sms * 8;
  multi_counters_init_kernel<<<m->num_sms * 4, 256, 0, s>>>(m->counters, num_graphs);
  if (L.total_vertices) {
    if (L.units) {
      multi_partition_kernel<<<grid, 256, 0, s>>>(M);
      multi_validate_edges_kernel<<<grid, 256, 0, s>>>(M);
    }
    multi_validate_exist_kernel<<<grid, 256, 0, s>>>(M);
    multi_validate_kernel<<<grid, 256, 0, s>>>(M);
  }
  MTRY(cudaGetLastError());
  MTRY(cudaMemcpyAsync(m->h_counters, m->counters, num_graphs * C_N * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s));
  m->checked_graphs = num_graphs;
  return MM_OK;
}

mm_status mm_multi_verdicts(mm_multi* m, uint64_t num_graphs, mm_verdict* h_out) {
  if (!m || (num_graphs && !h_out)) return mfail(MM_ERR_ARG, "null argument");
  if (num_graphs != m->checked_graphs)
    return mfail(MM_ERR_ARG, "%llu verdicts asked, the last check covered %llu graphs",
                 (unsigned long long)num_graphs, (unsigned long long)m->checked_graphs);
  for (uint64_t g = 0; g < num_graphs; ++g) {
    const unsigned long long* c = m->h_counters + g * C_N;
    mm_verdict v{};
    v.n_matched = c[C_MATCHED];
    v.n_pairs = c[C_PAIRS];
    v.n_bad_range = c[C_RANGE];
    v.n_asym = c[C_ASYM];
    v.n_nonedge = c[C_NONEDGE];
    v.n_uncovered = c[C_UNCOVERED];
    v.n_pairs_bad = 0;
    v.first_bad_vertex = c[C_FIRST_BAD];
    v.first_uncovered = c[C_FIRST_UNCOVERED];
    if (v.n_bad_range) v.flags |= MM_V_RANGE;
    if (v.n_asym) v.flags |= MM_V_ASYM;
    if (v.n_nonedge) v.flags |= MM_V_NONEDGE;
    if (v.n_uncovered) v.flags |= MM_V_UNCOVERED;
    h_out[g] = v;
  }
  return MM_OK;
}

mm_status mm_validate_multi(mm_multi* m, uint64_t num_graphs, const mm_graph_desc* h_descs,
                            mm_verdict* h_out, void* cuda_stream) {
  if (!m || (num_graphs && !h_out)) return mfail(MM_ERR_ARG, "null argument");
  mm_status st = mm_validate_multi_async(m, num_graphs, h_descs, cuda_stream);
  if (st != MM_OK) return st;
  MTRY(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)));
  return mm_multi_verdicts(m, num_graphs, h_out);
}

mm_status mm_multi_destroy(mm_multi* m) {
  if (!m) return MM_OK;
  for (TableSet* t : {&m->sweep, &m->check}) {
    if (t->staging_pending && t->staging_free) cudaEventSynchronize(t->staging_free);
    if (t->staging_free) cudaEventDestroy(t->staging_free);
    if (t->tables) cudaFree(t->tables);
    if (t->staging) cudaFreeHost(t->staging);
    if (t->part) cudaFree(t->part);
    if (t->gid) cudaFree(t->gid);
  }
  if (m->pool) cudaFree(m->pool);
  if (m->counters) cudaFree(m->counters);
  if (m->ctrl) cudaFree(m->ctrl);
  if (m->h_err) cudaFreeHost(m->h_err);
  if (m->h_counters) cudaFreeHost(m->h_counters);
  delete m;
  return MM_OK;
}

}  // extern "C"
