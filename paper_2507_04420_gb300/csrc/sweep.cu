// sweep.cu -- Skipper's single pass over the CSR entries on sm_103a.
//
// prepare_kernel: Algorithm 1 lines 3-4 (every vertex ACC, mate unmatched)
//   fused with the merge-path partition of rows + entries into equal work
//   units, the GPU form of the paper's contiguous blocks of consecutive
//   vertices with about equal edge counts, handed to threads with work
//   stealing (Section IV-C).
// sweep_kernel: Algorithm 1 lines 5-18.  Persistent warps take units from a
//   global counter (the paper's idle threads steal work; here every unit is
//   handed out on demand), in ascending order or in dispersed runs
//   (UnitOrder, state.cuh), and walk each with sweep_unit (walk.cuh): 32-row
//   windows whose row ends and row states are loaded in one step, matched
//   rows skipped without a load, unmatched entries read 128 at a time with
//   128-bit loads, filtered by the states of both endpoints, and the surviving
//   candidates of one row tried one lane at a time.
// serial kernels: one thread, rows in ascending order, neighbours in stored
//   order -- the sequential greedy order (Section II-B).
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "walk.cuh"

namespace skp {

namespace {

// Fill p[0, count) with `value`, except p[special] = special_value (special
// may be out of range): 128-bit stores for the aligned body, plain stores for
// the ragged ends.  The element `special` is written by the store covering it.
__device__ __forceinline__ void fill_words(uint32_t* p, uint64_t count, uint32_t value, uint64_t special,
                                           uint32_t special_value, uint64_t tid, uint64_t nthreads) {
  const uint64_t head = ((16u - (reinterpret_cast<uintptr_t>(p) & 15u)) & 15u) / 4u;
  const uint64_t h = head < count ? head : count;
  for (uint64_t i = tid; i < h; i += nthreads) p[i] = i == special ? special_value : value;
  const uint64_t body = (count - h) / 4;
  uint4* q = reinterpret_cast<uint4*>(p + h);
  for (uint64_t i = tid; i < body; i += nthreads) {
    const uint64_t e = h + 4 * i;
    uint4 v = make_uint4(value, value, value, value);
    if (special - e < 4) {
      const uint32_t k = (uint32_t)(special - e);
      if (k == 0) v.x = special_value; else if (k == 1) v.y = special_value;
      else if (k == 2) v.z = special_value; else v.w = special_value;
    }
    q[i] = v;
  }
  for (uint64_t i = h + 4 * body + tid; i < count; i += nthreads) p[i] = i == special ? special_value : value;
}

template <int kBits>
__global__ void prepare_kernel(SweepParams P, uint64_t* graph_pairs, uint64_t num_graphs) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n = P.n;
  const uint64_t none = ~0ull;
  if (kBits == 32) {
    fill_words(P.state, n, kWAcc, P.poison ? P.poison - 1 : none, kWRsvd, tid, nthreads);
  } else {
    constexpr uint64_t per = 32 / kBits;
    const uint64_t pv = P.poison ? P.poison - 1 : none;
    fill_words(P.state, packed_words(n, kBits), 0u, P.poison ? pv / per : none,
               P.poison ? kRsvd << ((pv % per) * kBits) : 0u, tid, nthreads);
    fill_words(P.mate, n, kNone, none, kNone, tid, nthreads);
  }
  const int64_t total = (int64_t)(n + P.nnz);
  for (uint64_t u = tid; u <= P.units; u += nthreads) {
    int64_t d = (int64_t)(u * P.grain);
    if (d > total) d = total;
    const int64_t rows = merge_path_rows(P.offsets, (int64_t)n, (int64_t)P.nnz, d);
    P.part[2 * u] = rows;
    P.part[2 * u + 1] = d - rows;
  }
  for (uint64_t g = tid; g < num_graphs && graph_pairs; g += nthreads) graph_pairs[g] = 0;
  if (P.stats && tid < kStCount) P.stats[tid] = 0ull;
  if (tid == 0) {
    *P.work = 0ull;
    *P.err = 0u;
  }
}

// Two register budgets: 40 registers a thread (3 blocks of 512 threads, 48
// warps per SM) by default; kLean compiles for 32 (4 blocks, 64 warps per SM,
// a few more spills), which hides more memory latency where the state array
// stays in L2.
template <class S, bool kStats = false, bool kSym = false, bool kSel = false, bool kTile = false,
          bool kLean = false>
__global__ void __launch_bounds__(512, kLean ? 4 : 3) sweep_kernel(SweepParams P) {
  const unsigned lane = threadIdx.x & 31u;
  const S s(P);
  const uint64_t pol = policy_evict_first();
  uint32_t phase = 0;   // parity of the warp's tile barrier (kTile)
  if (kTile) init_window_tile(lane);
  const UnitOrder order(P.units, P.disperse != 0, (uint64_t)gridDim.x * (blockDim.x >> 5));
  for (;;) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(P.work, 1ull);
    c = __shfl_sync(kFull, c, 0);
    if (c >= order.total) return;
    const uint64_t w = order.unit(c);
    if (w >= P.units) continue;
    const int64_t row0 = P.part[2 * w];
    const int64_t e_begin = P.part[2 * w + 1];
    const int64_t e_end = P.part[2 * w + 3];
    if (e_begin < e_end)
      sweep_unit<S, kStats, kSym, kSel, kTile>(s, P, row0, e_begin, e_end, lane, pol, &phase);
    if ((c & 15) == 0) {  // stop handing out work once an error is recorded
      uint32_t e = 0;
      if (lane == 0) e = ld_relaxed(P.err);
      if (__shfl_sync(kFull, e, 0) & kErrTimeout) return;
    }
  }
}

template <class S>
__global__ void serial_kernel(SweepParams P) {
  if (blockIdx.x == 0 && threadIdx.x == 0) serial_rows(S(P), P, 0, P.n);
}

template <class S>
__global__ void serial_batched_kernel(SweepParams P) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < P.num_graphs) {
    uint64_t r0 = (uint64_t)P.vbase[g], r1 = (uint64_t)P.vbase[g + 1];
    r1 = r1 < P.n ? r1 : P.n;  // rows past n do not exist
    if (r0 < r1) serial_rows(S(P), P, r0, r1);
  }
}

__global__ void graph_pairs_kernel(const uint32_t* __restrict__ mate,
                                   const int64_t* __restrict__ vbase, uint64_t num_graphs,
                                   uint64_t n, unsigned long long* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x; v0 < n; v0 += stride) {
    const uint64_t v = v0 + threadIdx.x;
    bool take = false;
    uint64_t g = 0;
    if (v < n) {
      const uint32_t m = mate[v];
      take = m != kNone && m < n && v < m;
      if (take) {  // graph of v: last g with vbase[g] <= v
        uint64_t lo = 0, hi = num_graphs;
        while (hi - lo > 1) {
          const uint64_t mid = (lo + hi) >> 1;
          if ((uint64_t)__ldg(vbase + mid) <= v) lo = mid; else hi = mid;
        }
        g = lo;
      }
    }
    const unsigned active = __ballot_sync(kFull, take);
    if (take) {
      const unsigned same = __match_any_sync(active, g);
      if ((threadIdx.x & 31) == (unsigned)(__ffs(same) - 1)) atomicAdd(out + g, (unsigned long long)__popc(same));
    }
  }
}

}  // namespace

// run F with the state type for `bits` (2, 8 or 32)
#define SKP_DISPATCH_STATE(bits, F) \
  ((bits) == 32 ? F(WordState, 32) : (bits) == 2 ? F(TwoBitState, 2) : F(ByteState, 8))
// the same for the packed layouts only (2 or 8)
#define SKP_DISPATCH_PACKED(bits, F) ((bits) == 2 ? F(TwoBitState, 2) : F(ByteState, 8))

int sweep_blocks_per_sm(int bits, int block_threads, bool lean) {
  int b = 0;
#define OCC(S, B)                                                                                       \
  (lean ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sweep_kernel<S, false, false, false, false, true>, \
                                                        block_threads, 0)                               \
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sweep_kernel<S>, block_threads, 0))
  cudaError_t e = SKP_DISPATCH_STATE(bits, OCC);
#undef OCC
  if (e != cudaSuccess || b < 1) return 1;
  return b;
}

bool sweep_lean(int bits, int block_threads, int blocks_per_sm, bool state_fits_l2) {
  if (blocks_per_sm > 0) return blocks_per_sm > sweep_blocks_per_sm(bits, block_threads, false);
  return state_fits_l2;
}

cudaError_t launch_prepare(const SweepParams& P, int bits, int grid, cudaStream_t s,
                           uint64_t* graph_pairs_zero, uint64_t num_graphs) {
#define L(S, B) (prepare_kernel<B><<<grid, 256, 0, s>>>(P, graph_pairs_zero, num_graphs), 0)
  SKP_DISPATCH_STATE(bits, L);
#undef L
  return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepParams& P, int bits, int grid, int block, cudaStream_t s) {
  if (block > 512 || block < 32 || block % 32) return cudaErrorInvalidValue;
  // instances: statistics or not, symmetric filter or not, selective id loads
  // or not (statistics instances load eagerly), staged windows or not (the
  // host side asks for them only for packed states over an aligned device CSR)
  if (P.tile && !P.stats && !P.sel && bits != 32) {
#define L(S, B) (P.sym ? (sweep_kernel<S, false, true, false, true><<<grid, block, 0, s>>>(P), 0) \
                       : (sweep_kernel<S, false, false, false, true><<<grid, block, 0, s>>>(P), 0))
    SKP_DISPATCH_PACKED(bits, L);
#undef L
  } else if (P.sel && !P.stats && P.sym) {
#define L(S, B) (sweep_kernel<S, false, true, true><<<grid, block, 0, s>>>(P), 0)
    SKP_DISPATCH_STATE(bits, L);
#undef L
  } else if (P.sel && !P.stats) {
#define L(S, B) (sweep_kernel<S, false, false, true><<<grid, block, 0, s>>>(P), 0)
    SKP_DISPATCH_STATE(bits, L);
#undef L
  } else if (P.stats && P.sym) {
#define L(S, B) (sweep_kernel<S, true, true><<<grid, block, 0, s>>>(P), 0)
    SKP_DISPATCH_STATE(bits, L);
#undef L
  } else if (P.stats) {
#define L(S, B) (sweep_kernel<S, true><<<grid, block, 0, s>>>(P), 0)
    SKP_DISPATCH_STATE(bits, L);
#undef L
  } else if (P.sym) {
#define L(S, B) (P.lean ? (sweep_kernel<S, false, true, false, false, true><<<grid, block, 0, s>>>(P), 0) \
                        : (sweep_kernel<S, false, true><<<grid, block, 0, s>>>(P), 0))
    SKP_DISPATCH_STATE(bits, L);
#undef L
  } else {
#define L(S, B) (P.lean ? (sweep_kernel<S, false, false, false, false, true><<<grid, block, 0, s>>>(P), 0) \
                        : (sweep_kernel<S><<<grid, block, 0, s>>>(P), 0))
    SKP_DISPATCH_STATE(bits, L);
#undef L
  }
  return cudaGetLastError();
}

cudaError_t launch_serial(const SweepParams& P, int bits, cudaStream_t s) {
#define L(S, B) (serial_kernel<S><<<1, 1, 0, s>>>(P), 0)
  SKP_DISPATCH_STATE(bits, L);
#undef L
  return cudaGetLastError();
}

cudaError_t launch_serial_batched(const SweepParams& P, int bits, cudaStream_t s) {
  const unsigned grid = (unsigned)((P.num_graphs + 127) / 128);
  if (grid == 0) return cudaSuccess;
#define L(S, B) (serial_batched_kernel<S><<<grid, 128, 0, s>>>(P), 0)
  SKP_DISPATCH_STATE(bits, L);
#undef L
  return cudaGetLastError();
}

void get_batched_kernels(int bits, bool serial, bool sym, bool lean, const void** prepare,
                         const void** sweep, const void** pairs) {
#define PK(S, B) (const void*)prepare_kernel<B>
#define SB(S, B) (const void*)serial_batched_kernel<S>
#define SW(S, B) (lean ? (const void*)sweep_kernel<S, false, false, false, false, true> : (const void*)sweep_kernel<S>)
#define SY(S, B) (lean ? (const void*)sweep_kernel<S, false, true, false, false, true> \
                       : (const void*)sweep_kernel<S, false, true>)
  *prepare = SKP_DISPATCH_STATE(bits, PK);
  *sweep = serial ? SKP_DISPATCH_STATE(bits, SB)
                  : sym ? SKP_DISPATCH_STATE(bits, SY) : SKP_DISPATCH_STATE(bits, SW);
#undef PK
#undef SB
#undef SW
#undef SY
  *pairs = (const void*)graph_pairs_kernel;
}

cudaError_t launch_graph_pairs(const uint32_t* mate, const int64_t* vbase, uint64_t num_graphs,
                               uint64_t n, uint64_t* graph_pairs, int grid, cudaStream_t s) {
  if (n == 0 || num_graphs == 0) return cudaSuccess;
  graph_pairs_kernel<<<grid, 256, 0, s>>>(mate, vbase, num_graphs, n,
                                          reinterpret_cast<unsigned long long*>(graph_pairs));
  return cudaGetLastError();
}

}  // namespace skp
