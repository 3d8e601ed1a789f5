// sweep.cu -- Skipper's single pass over the CSR entries on sm_103a.
//
// prepare_kernel: Algorithm 1 lines 3-4 (every vertex ACC, mate unmatched)
//   fused with the merge-path partition of rows + entries into equal work
//   units, the GPU form of the paper's blocks of consecutive vertices with
//   about equal edge counts (Section IV-C, "thread-dispersed
//   locality-preserving" scheduling).
// sweep_kernel: Algorithm 1 lines 5-18.  Persistent warps take units from a
//   global counter (the paper's idle threads steal work; here every unit is
//   handed out on demand).  A warp walks its unit in chunks of up to 128
//   entries: 32 lanes x one 128-bit load of four neighbour ids.  Before a chunk
//   is read, the state of the row vertex at its head is checked and a matched
//   row is left at once, so the remaining neighbour ids of a matched source are
//   never loaded.  Within a chunk every lane filters its entries by the states
//   of both endpoints; the surviving candidates of one row are tried one at a
//   time (lowest lane first), so the lanes of a warp never race each other for
//   the same row vertex, while candidates of different rows proceed together.
// serial kernels: one thread, rows in ascending order, neighbours in stored
//   order -- the sequential greedy order (Section II-B).
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace skp {

namespace {

// a[j] for a run-time j without local-memory indexing
__device__ __forceinline__ uint32_t pick4(const uint32_t (&a)[4], int j) {
  uint32_t r = a[0];
#pragma unroll
  for (int i = 1; i < 4; ++i) r = j == i ? a[i] : r;
  return r;
}

// Merge-path split of diagonal d over the row ends offsets[1..n] and the entry
// indices 0..nnz-1 (a row end equal to an entry index is taken first): returns
// the number of rows finished before the split; entry index = d - rows.
__device__ __forceinline__ int64_t merge_path_rows(const int64_t* offsets, int64_t n, int64_t nnz,
                                                   int64_t d) {
  int64_t lo = d - nnz > 0 ? d - nnz : 0;
  int64_t hi = d < n ? d : n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (offsets[mid + 1] <= d - mid - 1)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

template <bool kWord>
__global__ void prepare_kernel(SweepParams P, uint64_t* graph_pairs, uint64_t num_graphs) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n = P.n;
  if (kWord) {
    for (uint64_t v = tid; v < n; v += nthreads)
      P.state[v] = (P.poison && v == P.poison - 1) ? kWRsvd : kWAcc;
  } else {
    const uint64_t nwords = (n + 3) >> 2;
    for (uint64_t i = tid; i < nwords; i += nthreads) {
      uint32_t w = 0u;  // four ACC bytes
      if (P.poison && ((P.poison - 1) >> 2) == i) w = kRsvd << (((P.poison - 1) & 3u) << 3);
      P.state[i] = w;
    }
    for (uint64_t v = tid; v < n; v += nthreads) P.mate[v] = kNone;
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
  if (tid == 0) {
    *P.work = 0ull;
    *P.err = 0u;
  }
}

// number of lanes k whose ascending value rel_k is <= p (32-bit); the caller
// guarantees rel_31 > p for the lanes whose answer it uses.
__device__ __forceinline__ int count_le(int rel, int p) {
  int c = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const int v = __shfl_sync(kFull, rel, c + step - 1);
    if (v <= p) c += step;
  }
  return c;
}

// One work unit: entries [pos, e_end), the first of which lies in row >= row0.
//
// The warp keeps a window of 32 consecutive rows: lane k holds the end offset
// of row wbase+k and the word holding that row vertex's state, both loaded in
// one coalesced step, and `mchd` has bit k set when row wbase+k is known to be
// matched.  Matched rows are jumped over with bit arithmetic, so a matched
// source costs no load of its own (Skipper leaves the rest of a matched row;
// SGMM does the same in CSR order, Section II-B).  The unmatched entries are
// read in chunks of up to 128 (one aligned 128-bit load per lane); the state
// of the row at the head of each chunk is re-read alongside, so a long row
// matched by another warp is left after at most one more chunk.
template <class S>
__device__ __forceinline__ void sweep_unit(const S& s, const SweepParams& P, int64_t row0,
                                           int64_t pos, const int64_t e_end, const unsigned lane,
                                           const uint64_t pol_stream) {
  const uint32_t n32 = (uint32_t)P.n;
  int64_t wbase = row0;
  int64_t my_end;
  uint32_t my_st;
  unsigned mchd;
  {
    const int64_t r = wbase + lane;
    const bool in = r < (int64_t)P.n;
    my_end = in ? __ldg(P.offsets + r + 1) : INT64_MAX;
    my_st = in ? s.peek((uint32_t)r) : 0u;
    mchd = __ballot_sync(kFull, !in || S::matched(my_st, (uint32_t)r));  // rows past n hold no entries
  }
  while (pos < e_end) {
    // rows of the window with entries at or after pos that are not known matched
    const unsigned open = __ballot_sync(kFull, my_end > pos) & ~mchd;
    if (open == 0u) {  // the window is exhausted: continue after its last row
      const int64_t win_end = __shfl_sync(kFull, my_end, 31);
      if (win_end >= e_end) return;
      if (win_end > pos) pos = win_end;
      wbase += 32;
      const int64_t r = wbase + lane;
      const bool in = r < (int64_t)P.n;
      my_end = in ? __ldg(P.offsets + r + 1) : INT64_MAX;
      my_st = in ? s.peek((uint32_t)r) : 0u;
      mchd = __ballot_sync(kFull, !in || S::matched(my_st, (uint32_t)r));
      continue;
    }
    const int k1 = __ffs(open) - 1;
    if (k1 > 0) {  // row k1 starts where row k1-1 ends
      const int64_t st = __shfl_sync(kFull, my_end, k1 - 1);
      if (st > pos) pos = st;
    }
    if (pos >= e_end) return;
    const int64_t win_end = __shfl_sync(kFull, my_end, 31);
    const int64_t base = pos & ~(int64_t)3;
    int64_t cend = base + 128;
    if (cend > e_end) cend = e_end;
    if (cend > win_end) cend = win_end;
    // chunk-relative 32-bit coordinates: entry base+p, p in [lo_r, hi_r)
    const int lo_r = (int)(pos - base);
    const int hi_r = (int)(cend - base);
    const int64_t rel64 = my_end - base;
    const int rel = rel64 < 0 ? -1 : (rel64 > 129 ? 129 : (int)rel64);

    // neighbour ids (one aligned 128-bit load per lane) and, in parallel, a
    // fresh read of the head row's state
    const int p0 = 4 * (int)lane;
    const int64_t e0 = base + p0;
    uint32_t y[4] = {0u, 0u, 0u, 0u};
    if (p0 < hi_r) {
      if (e0 + 4 <= (int64_t)P.nnz) {
        const uint4 q = ld_stream_v4(P.nbrs + e0, pol_stream);
        y[0] = q.x; y[1] = q.y; y[2] = q.z; y[3] = q.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (e0 + j < (int64_t)P.nnz) y[j] = ld_stream(P.nbrs + e0 + j, pol_stream);
      }
    }
    const uint32_t x1 = (uint32_t)(wbase + k1);
    uint32_t head = 0;
    if (lane == 0) head = s.peek(x1);
    head = __shfl_sync(kFull, head, 0);
    if (S::matched(head, x1)) mchd |= 1u << k1;
    if (lane == (unsigned)k1) my_st = head;

    // row of each entry within the window
    int k[4];
    k[0] = count_le(rel, p0);
    k[3] = count_le(rel, p0 + 3);
    if (__any_sync(kFull, k[0] != k[3])) {
      k[1] = count_le(rel, p0 + 1);
      k[2] = count_le(rel, p0 + 2);
    } else {
      k[1] = k[0];
      k[2] = k[0];
    }
    // words holding the row states, from the window snapshot
    uint32_t rx[4], xs[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      rx[j] = __shfl_sync(kFull, my_st, k[j] & 31);
      xs[j] = (uint32_t)(wbase + k[j]);
    }

    // filter (the line-10 read): candidates have both endpoints unmatched
    bool want[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = p0 + j;
      want[j] = p >= lo_r && p < hi_r && !(mchd >> (k[j] & 31) & 1u) && !S::matched(rx[j], xs[j]) &&
                y[j] != xs[j];
      if (want[j] && y[j] >= n32) {
        atomicOr(P.err, kErrBadId);
        want[j] = false;
      }
    }
    uint32_t ry[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (want[j]) ry[j] = s.peek(y[j]);
    uint32_t cand = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (want[j] && !S::matched(ry[j], y[j])) cand |= 1u << j;

    // resolve candidates: per row, one lane at a time
    for (;;) {
      const bool have = cand != 0u;
      if (!__any_sync(kFull, have)) break;
      const int j = have ? __ffs(cand) - 1 : 0;
      const uint32_t key = have ? pick4(xs, j) : kNone;
      const unsigned peers = __match_any_sync(kFull, key);
      const int leader = __ffs(peers) - 1;
      unsigned done = 0u;
      if (have && (int)lane == leader) {
        cand &= ~(1u << j);
        if (resolve_edge(s, key, pick4(y, j), pick4(rx, j), pick4(ry, j), P))
          done = 1u << (key - (uint32_t)wbase);
      }
      done = __reduce_or_sync(kFull, done);  // rows that are now matched
      mchd |= done;
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
        if (done >> (k[jj] & 31) & 1u) cand &= ~(1u << jj);
    }
    pos = cend;
  }
}

template <class S>
__global__ void __launch_bounds__(512, 3) sweep_kernel(SweepParams P) {
  const unsigned lane = threadIdx.x & 31u;
  const S s(P);
  const uint64_t pol = policy_evict_first();
  for (;;) {
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(P.work, 1ull);
    w = __shfl_sync(kFull, w, 0);
    if (w >= P.units) return;
    const int64_t row0 = P.part[2 * w];
    const int64_t e_begin = P.part[2 * w + 1];
    const int64_t e_end = P.part[2 * w + 3];
    if (e_begin < e_end) sweep_unit(s, P, row0, e_begin, e_end, lane, pol);
    if ((w & 15) == 0) {  // stop handing out work once an error is recorded
      uint32_t e = 0;
      if (lane == 0) e = ld_relaxed(P.err);
      if (__shfl_sync(kFull, e, 0) & kErrTimeout) return;
    }
  }
}

template <class S>
__device__ __forceinline__ void serial_rows(const S& s, const SweepParams& P, uint64_t r0,
                                            uint64_t r1) {
  for (uint64_t x = r0; x < r1; ++x) {
    if (S::matched(s.raw((uint32_t)x), (uint32_t)x)) continue;
    for (int64_t i = P.offsets[x]; i < P.offsets[x + 1]; ++i) {
      const uint32_t y = P.nbrs[i];
      if (y >= P.n) {
        atomicOr(P.err, kErrBadId);
        continue;
      }
      if (y == x) continue;
      if (resolve_edge(s, (uint32_t)x, y, s.raw((uint32_t)x), s.raw(y), P)) break;
      if (ld_relaxed(P.err) & kErrTimeout) return;
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

int sweep_blocks_per_sm(bool word, int block_threads) {
  int b = 0;
  cudaError_t e = word ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sweep_kernel<WordState>, block_threads, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sweep_kernel<ByteState>, block_threads, 0);
  if (e != cudaSuccess || b < 1) return 1;
  return b;
}

cudaError_t launch_prepare(const SweepParams& P, bool word, int grid, cudaStream_t s,
                           uint64_t* graph_pairs_zero, uint64_t num_graphs) {
  if (word)
    prepare_kernel<true><<<grid, 256, 0, s>>>(P, graph_pairs_zero, num_graphs);
  else
    prepare_kernel<false><<<grid, 256, 0, s>>>(P, graph_pairs_zero, num_graphs);
  return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepParams& P, bool word, int grid, int block, cudaStream_t s) {
  if (block > 512 || block < 32 || block % 32) return cudaErrorInvalidValue;
  if (word)
    sweep_kernel<WordState><<<grid, block, 0, s>>>(P);
  else
    sweep_kernel<ByteState><<<grid, block, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_serial(const SweepParams& P, bool word, cudaStream_t s) {
  if (word)
    serial_kernel<WordState><<<1, 1, 0, s>>>(P);
  else
    serial_kernel<ByteState><<<1, 1, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_serial_batched(const SweepParams& P, bool word, cudaStream_t s) {
  const unsigned grid = (unsigned)((P.num_graphs + 127) / 128);
  if (grid == 0) return cudaSuccess;
  if (word)
    serial_batched_kernel<WordState><<<grid, 128, 0, s>>>(P);
  else
    serial_batched_kernel<ByteState><<<grid, 128, 0, s>>>(P);
  return cudaGetLastError();
}

void get_batched_kernels(bool word, bool serial, const void** prepare, const void** sweep,
                         const void** pairs) {
  *prepare = word ? (const void*)prepare_kernel<true> : (const void*)prepare_kernel<false>;
  if (serial)
    *sweep = word ? (const void*)serial_batched_kernel<WordState>
                  : (const void*)serial_batched_kernel<ByteState>;
  else
    *sweep = word ? (const void*)sweep_kernel<WordState> : (const void*)sweep_kernel<ByteState>;
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
