// batch.cu -- batched Skipper with a partition of its own for every member
// graph: the work units of a graph never cross into the next one, their
// number per graph may be capped (warps per graph), and the member graphs may
// hold local ids (MM_BATCH_LOCAL_IDS), so a batch can hold more than 2^32
// vertices in all while each graph keeps uint32 ids.
//
// Every table the launch needs is computed on the device from the caller's
// vbase / ebase arrays (batch_plan_kernel: units and state words per graph,
// scanned; batch_prepare_kernel: Algorithm 1 lines 3-4 and the merge-path
// split of each graph), so a CUDA graph of these launches replays on new
// contents of the same buffers without host work.  A unit is walked by the
// single-graph walk (walk.cuh, Algorithm 1 lines 5-18) on a view of its
// graph: with local ids the view's row ends start at the graph's first row
// (their values stay global entry indices, which the walk only compares and
// loads through), its states and mates start at the graph's own base.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "walk.cuh"
#include "checkwalk.cuh"

namespace skp {
namespace {

constexpr int kPlanThreads = 1024;

// last g < G with base[g] <= x (base ascending, base[0] = 0 <= x < base[G])
__device__ __forceinline__ uint64_t last_at_or_below(const int64_t* base, uint64_t G, uint64_t x) {
  uint64_t lo = 0, hi = G;
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if ((uint64_t)__ldg(base + mid) <= x) lo = mid; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ uint64_t last_at_or_below_u(const uint64_t* base, uint64_t G, uint64_t x) {
  uint64_t lo = 0, hi = G;
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (base[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// Merge-path split of diagonal d of one graph whose row ends are
// offsets[1..n] - e0 (the graph's entries start at global index e0).
__device__ __forceinline__ int64_t merge_path_rows_at(const int64_t* offsets, int64_t n, int64_t nnz,
                                                      int64_t d, int64_t e0) {
  int64_t lo = d - nnz > 0 ? d - nnz : 0;
  int64_t hi = d < n ? d : n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (offsets[mid + 1] - e0 <= d - mid - 1)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// The view of graph g that the walk runs on.
template <bool kLocal, bool kWord>
__device__ __forceinline__ SweepParams graph_view(const BatchParams& B, uint64_t g) {
  SweepParams P = B.P;
  if (kLocal) {
    const int64_t vb = B.vbase[g];
    P.n = (uint64_t)(B.vbase[g + 1] - vb);
    P.offsets = B.P.offsets + vb;
    P.mate = B.P.mate + vb;
    P.state = kWord ? P.mate : B.P.state + B.sbase[g];
  }
  return P;
}

// Units (and, with local ids in a packed layout, state words) of every graph,
// scanned into ubase / sbase by one block of kPlanThreads threads.
template <int kBits>
__global__ void __launch_bounds__(kPlanThreads) batch_plan_kernel(BatchParams B) {
  __shared__ uint64_t wu[32], ws[32];
  __shared__ uint64_t carry_u, carry_s;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_u = carry_s = 0;
  __syncthreads();
  const uint64_t G = B.num_graphs;
  for (uint64_t base = 0; base < G; base += kPlanThreads) {
    const uint64_t g = base + threadIdx.x;
    uint64_t u = 0, w = 0;
    if (g < G) {
      const uint64_t ng = (uint64_t)(B.vbase[g + 1] - B.vbase[g]);
      const uint64_t eg = (uint64_t)(B.ebase[g + 1] - B.ebase[g]);
      u = (ng + eg + B.grain - 1) / B.grain;
      if (B.wpg && u > B.wpg) u = B.wpg;
      if (B.local && kBits != 32) w = packed_words(ng, kBits);
    }
    uint64_t iu = u, iw = w;   // inclusive scan within the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t a = __shfl_up_sync(kFull, iu, d), b = __shfl_up_sync(kFull, iw, d);
      if ((int)lane >= d) {
        iu += a;
        iw += b;
      }
    }
    if (lane == 31) {
      wu[warp] = iu;
      ws[warp] = iw;
    }
    __syncthreads();
    if (warp == 0) {           // scan of the warp totals
      uint64_t x = wu[lane], y = ws[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t a = __shfl_up_sync(kFull, x, d), b = __shfl_up_sync(kFull, y, d);
        if ((int)lane >= d) {
          x += a;
          y += b;
        }
      }
      wu[lane] = x;
      ws[lane] = y;
    }
    __syncthreads();
    if (g < G) {
      B.ubase[g] = carry_u + (warp ? wu[warp - 1] : 0) + iu - u;
      B.sbase[g] = carry_s + (warp ? ws[warp - 1] : 0) + iw - w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry_u += wu[31];
      carry_s += ws[31];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    B.ubase[G] = carry_u;
    B.sbase[G] = carry_s;
    B.totals[0] = carry_u;
    B.totals[1] = carry_s;
  }
}

// p[0, count) := value (128-bit stores for the aligned body)
__device__ __forceinline__ void fill(uint32_t* p, uint64_t count, uint32_t value, uint64_t tid,
                                     uint64_t nthreads) {
  const uint64_t head = ((16u - (reinterpret_cast<uintptr_t>(p) & 15u)) & 15u) / 4u;
  const uint64_t h = head < count ? head : count;
  for (uint64_t i = tid; i < h; i += nthreads) p[i] = value;
  const uint64_t body = (count - h) / 4;
  uint4* q = reinterpret_cast<uint4*>(p + h);
  for (uint64_t i = tid; i < body; i += nthreads) q[i] = make_uint4(value, value, value, value);
  for (uint64_t i = h + 4 * body + tid; i < count; i += nthreads) p[i] = value;
}

// Algorithm 1 lines 3-4 (every vertex ACC, mate unmatched) and the merge-path
// units of every graph (after batch_plan_kernel).  With `states` false only
// the units are made (the checker's partition).
template <int kBits>
__global__ void batch_prepare_kernel(BatchParams B, int states) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n = B.P.n;
  const uint64_t G = B.num_graphs;
  if (states) {
    if (kBits == 32) {
      fill(B.P.mate, n, kWAcc, tid, nthreads);
    } else {
      fill(B.P.state, B.local ? B.totals[1] : packed_words(n, kBits), 0u, tid, nthreads);
      fill(B.P.mate, n, kNone, tid, nthreads);
    }
  }
  const uint64_t units = B.totals[0];
  for (uint64_t u = tid; u < units; u += nthreads) {
    const uint64_t g = last_at_or_below_u(B.ubase, G, u);
    const int64_t vb = B.vbase[g], eb = B.ebase[g];
    const int64_t ng = B.vbase[g + 1] - vb, eg = B.ebase[g + 1] - eb;
    const uint64_t ug = B.ubase[g + 1] - B.ubase[g];
    const int64_t items = ng + eg;
    const int64_t size = (items + (int64_t)ug - 1) / (int64_t)ug;   // items per unit of this graph
    int64_t d = (int64_t)(u - B.ubase[g]) * size;
    if (d > items) d = items;
    const int64_t rows = merge_path_rows_at(B.P.offsets + vb, ng, eg, d, eb);
    B.part[2 * u] = B.local ? rows : vb + rows;
    B.part[2 * u + 1] = eb + d - rows;
    B.gid[u] = (uint32_t)g;
  }
  if (states) {
    for (uint64_t g = tid; g < G && B.graph_pairs; g += nthreads) B.graph_pairs[g] = 0;
    if (tid == 0) {
      *B.P.work = 0ull;
      *B.P.err = 0u;
    }
  }
}

template <class S, bool kLocal, bool kSym, bool kLean>
__global__ void __launch_bounds__(512, kLean ? 4 : 3) batch_sweep_kernel(BatchParams B) {
  constexpr bool kWord = S::kPerWord == 1;
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t pol = policy_evict_first();
  const uint64_t units = B.totals[0];
  const UnitOrder order(units, B.P.disperse != 0, (uint64_t)gridDim.x * (blockDim.x >> 5));
  for (;;) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(B.P.work, 1ull);
    c = __shfl_sync(kFull, c, 0);
    if (c >= order.total) return;
    const uint64_t w = order.unit(c);
    if (w >= units) continue;
    const uint32_t g = B.gid[w];
    const SweepParams P = graph_view<kLocal, kWord>(B, g);
    const int64_t row0 = B.part[2 * w];
    const int64_t e_begin = B.part[2 * w + 1];
    const int64_t e_end = (w + 1 < units && B.gid[w + 1] == g) ? B.part[2 * w + 3] : B.ebase[g + 1];
    if (e_begin < e_end) sweep_unit<S, false, kSym>(S(P), P, row0, e_begin, e_end, lane, pol);
    if ((c & 15) == 0) {  // stop handing out work once an error is recorded
      uint32_t e = 0;
      if (lane == 0) e = ld_relaxed(B.P.err);
      if (__shfl_sync(kFull, e, 0) & kErrTimeout) return;
    }
  }
}

// One thread per graph, rows in ascending order, neighbours in stored order:
// sequential greedy MM on every graph (Section II-B).
template <class S, bool kLocal>
__global__ void batch_serial_kernel(BatchParams B) {
  constexpr bool kWord = S::kPerWord == 1;
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B.num_graphs) return;
  const SweepParams P = graph_view<kLocal, kWord>(B, g);
  if (kLocal)
    serial_rows(S(P), P, 0, P.n);
  else
    serial_rows(S(P), P, (uint64_t)B.vbase[g], (uint64_t)B.vbase[g + 1]);
}

// Matched pairs per graph: vertex i of the batch, in graph g, counts when it
// is the lower end of its pair.
template <bool kLocal>
__global__ void batch_pairs_kernel(BatchParams B) {
  const uint64_t n = B.P.n, G = B.num_graphs;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const uint64_t i = i0 + threadIdx.x;
    bool take = false;
    uint64_t g = 0;
    if (i < n) {
      const uint32_t m = B.P.mate[i];
      if (m != kNone) {
        g = last_at_or_below(B.vbase, G, i);
        const uint64_t vb = (uint64_t)B.vbase[g];
        take = kLocal ? (m < (uint64_t)B.vbase[g + 1] - vb && i - vb < m) : (m < n && i < m);
      }
    }
    const unsigned active = __ballot_sync(kFull, take);
    if (take) {
      const unsigned same = __match_any_sync(active, g);
      if ((threadIdx.x & 31) == (unsigned)(__ffs(same) - 1))
        atomicAdd(reinterpret_cast<unsigned long long*>(B.graph_pairs) + g, (unsigned long long)__popc(same));
    }
  }
}

// ---- the exact checker over a batch (Section II-B), one verdict for all
// member graphs; vertex and entry indices are the batch's (global) ones ----
enum { BC_MATCHED = 0, BC_PAIRS, BC_RANGE, BC_ASYM, BC_NONEDGE, BC_UNCOVERED, BC_PAIRS_BAD,
       BC_FIRST_BAD, BC_FIRST_UNCOVERED, BC_N };

__global__ void batch_check_init_kernel(unsigned long long* c) {
  if (threadIdx.x < BC_N) c[threadIdx.x] = threadIdx.x >= BC_FIRST_BAD ? ~0ull : 0ull;
}

// edge pass: the uncovered entries of every unit of every graph
template <bool kLocal>
__global__ void batch_check_edges_kernel(BatchParams B, unsigned long long* c) {
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t units = B.totals[0];
  unsigned long long unc = 0, first = ~0ull;
  for (uint64_t u = warp; u < units; u += nwarps) {
    const uint32_t g = B.gid[u];
    const SweepParams P = graph_view<kLocal, true>(B, g);
    const int64_t e0 = B.part[2 * u + 1];
    const int64_t e1 = (u + 1 < units && B.gid[u + 1] == g) ? B.part[2 * u + 3] : B.ebase[g + 1];
    if (e0 < e1) check_unit(P.offsets, P.nbrs, P.n, P.nnz, P.mate, B.part[2 * u], e0, e1, lane, unc, first);
  }
  unc = warp_sum64(unc);
  first = warp_min64(first);
  if (lane == 0) {
    if (unc) atomicAdd(c + BC_UNCOVERED, unc);
    if (first != ~0ull) atomicMin(c + BC_FIRST_UNCOVERED, first);
  }
}

// vertex pass (range, symmetry, pairs) and existence pass (the named partner
// shares an edge, stored in either row, the shorter row searched first), one
// warp per 32 consecutive vertices of the batch
template <bool kLocal>
__global__ void batch_check_vertices_kernel(BatchParams B, unsigned long long* c) {
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t N = B.P.n, G = B.num_graphs;
  unsigned long long matched = 0, pairs = 0, range = 0, asym = 0, nonedge = 0, first_bad = ~0ull;
  for (uint64_t w0 = warp * 32; w0 < N; w0 += nwarps * 32) {
    const uint64_t i = w0 + lane;
    uint64_t g = 0, vb = 0, ng = N;
    uint32_t v = 0, m = kNone;
    bool valid = false, sym = false;
    if (i < N) {
      if (kLocal) {
        g = last_at_or_below(B.vbase, G, i);
        vb = (uint64_t)B.vbase[g];
        ng = (uint64_t)B.vbase[g + 1] - vb;
      }
      v = (uint32_t)(i - vb);
      m = B.P.mate[i];
      if (m != kNone) {
        if (m >= ng || m == v) {
          ++range;
          if (i < first_bad) first_bad = i;
        } else {
          ++matched;
          valid = true;
          sym = B.P.mate[vb + m] == v;
          if (!sym) {
            ++asym;
            if (i < first_bad) first_bad = i;
          } else if (v < m) {
            ++pairs;
          }
        }
      }
    }
    unsigned todo = __ballot_sync(kFull, valid && !(sym && m < v));
    while (todo) {
      const int j = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint64_t vbj = __shfl_sync(kFull, vb, j);
      const uint32_t vj = __shfl_sync(kFull, v, j), mj = __shfl_sync(kFull, m, j);
      const bool sj = __shfl_sync(kFull, sym ? 1u : 0u, j) != 0u;
      const int64_t* off = B.P.offsets + (kLocal ? vbj : 0);
      const int64_t dv = off[vj + 1] - off[vj];
      const int64_t dm = off[mj + 1] - off[mj];
      const bool v_first = dv <= dm;  // the shorter row first
      bool hit = warp_row_has(off, B.P.nbrs, v_first ? vj : mj, v_first ? mj : vj, lane);
      if (!hit) hit = warp_row_has(off, B.P.nbrs, v_first ? mj : vj, v_first ? vj : mj, lane);
      if (!hit && lane == 0) {
        nonedge += sj ? 2 : 1;
        if (vbj + vj < first_bad) first_bad = vbj + vj;
      }
    }
  }
  matched = warp_sum64(matched);
  pairs = warp_sum64(pairs);
  range = warp_sum64(range);
  asym = warp_sum64(asym);
  nonedge = warp_sum64(nonedge);
  first_bad = warp_min64(first_bad);
  if (lane == 0) {
    if (matched) atomicAdd(c + BC_MATCHED, matched);
    if (pairs) atomicAdd(c + BC_PAIRS, pairs);
    if (range) atomicAdd(c + BC_RANGE, range);
    if (asym) atomicAdd(c + BC_ASYM, asym);
    if (nonedge) atomicAdd(c + BC_NONEDGE, nonedge);
    if (first_bad != ~0ull) atomicMin(c + BC_FIRST_BAD, first_bad);
  }
}

}  // namespace

#define SKP_BATCH_STATE(bits, F) \
  ((bits) == 32 ? F(WordState, 32) : (bits) == 2 ? F(TwoBitState, 2) : F(ByteState, 8))

void get_batch_kernels(int bits, bool local, bool serial, bool sym, bool lean, BatchKernels* k) {
#define PL(S, B) (const void*)batch_plan_kernel<B>
#define PR(S, B) (const void*)batch_prepare_kernel<B>
  k->plan = SKP_BATCH_STATE(bits, PL);
  k->prepare = SKP_BATCH_STATE(bits, PR);
#undef PL
#undef PR
  if (serial) {
#define SE(S, B) (local ? (const void*)batch_serial_kernel<S, true> : (const void*)batch_serial_kernel<S, false>)
    k->sweep = SKP_BATCH_STATE(bits, SE);
#undef SE
  } else {
#define SWL(S, L)                                                                           \
  (local ? (sym ? (const void*)batch_sweep_kernel<S, true, true, L> : (const void*)batch_sweep_kernel<S, true, false, L>) \
         : (sym ? (const void*)batch_sweep_kernel<S, false, true, L> : (const void*)batch_sweep_kernel<S, false, false, L>))
#define SW(S, B) (lean ? SWL(S, true) : SWL(S, false))
    k->sweep = SKP_BATCH_STATE(bits, SW);
#undef SW
#undef SWL
  }
  k->pairs = local ? (const void*)batch_pairs_kernel<true> : (const void*)batch_pairs_kernel<false>;
}

int batch_sweep_blocks_per_sm(int bits, bool local, bool sym, bool lean, int block_threads) {
  BatchKernels k{};
  get_batch_kernels(bits, local, false, sym, lean, &k);
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k.sweep, block_threads, 0) != cudaSuccess || b < 1)
    return 1;
  return b;
}

// The checker over a batch: partition every graph with the checker's grain
// (no state is touched), then the edge pass and the vertex pass.
cudaError_t launch_validate_batch(const BatchParams& B0, unsigned long long* counters, int grid,
                                  cudaStream_t s) {
  BatchParams B = B0;
  B.grain = kCheckGrain;
  B.wpg = 0;
  batch_check_init_kernel<<<1, 32, 0, s>>>(counters);
  batch_plan_kernel<32><<<1, kPlanThreads, 0, s>>>(B);
  batch_prepare_kernel<32><<<grid, 256, 0, s>>>(B, 0);
  if (B.local) {
    batch_check_edges_kernel<true><<<grid, 256, 0, s>>>(B, counters);
    batch_check_vertices_kernel<true><<<grid, 256, 0, s>>>(B, counters);
  } else {
    batch_check_edges_kernel<false><<<grid, 256, 0, s>>>(B, counters);
    batch_check_vertices_kernel<false><<<grid, 256, 0, s>>>(B, counters);
  }
  return cudaGetLastError();
}

int batch_plan_threads() { return kPlanThreads; }

}  // namespace skp
