// check.cu -- CSR input check, the exact maximal-matching checker and the
// ordered pair-list compaction, on the device.
//
// The checker follows the validation rule of Section II-B (every edge touches
// an output edge; no two output edges share an endpoint) with the counting
// rules stated in skipper.h, so its verdict can be compared field by field
// with a host checker.  Counters are aggregated per warp and added with 64-bit
// atomics; "first offender" fields take the minimum with atomicMin, so every
// field is independent of thread timing.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "checkwalk.cuh"
#include "walk.cuh"

namespace skp {

namespace {

enum { C_MATCHED = 0, C_PAIRS, C_RANGE, C_ASYM, C_NONEDGE, C_UNCOVERED, C_PAIRS_BAD,
       C_FIRST_BAD, C_FIRST_UNCOVERED, C_COUNT };

__global__ void zero_u64_kernel(unsigned long long* p, uint64_t words, unsigned long long v) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
       i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void zero_u32_kernel(uint32_t* p, uint64_t words) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
       i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = 0u;
}

__global__ void csr_check_kernel(uint64_t n, uint64_t nnz, const int64_t* __restrict__ offsets,
                                 const uint32_t* __restrict__ nbrs, unsigned long long* bad) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long local = 0;
  if (tid == 0 && (offsets[0] != 0 || offsets[n] != (int64_t)nnz)) ++local;
  for (uint64_t i = tid; i < n; i += stride)
    if (offsets[i] > offsets[i + 1]) ++local;
  for (uint64_t i = tid; i < nnz; i += stride)
    if (nbrs[i] >= n) ++local;
  if (local) atomicAdd(bad, local);
}

// edge-list input: every endpoint id < n
__global__ void coo_check_kernel(uint64_t n, uint64_t m, const uint32_t* __restrict__ src,
                                 const uint32_t* __restrict__ dst, unsigned long long* bad) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long local = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
    local += (src[i] >= n) + (dst[i] >= n);
  if (local) atomicAdd(bad, local);
}

__device__ __forceinline__ void warp_add(unsigned long long* c, uint32_t v) {
  const uint32_t s = __reduce_add_sync(kFull, v);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(c, (unsigned long long)s);
}

// Merge-path split of rows + entries into units of `grain` items (the same
// split the sweep uses), for the checker's edge pass.
__global__ void check_partition_kernel(uint64_t n, uint64_t nnz, const int64_t* __restrict__ offsets,
                                       uint64_t grain, uint64_t units, int64_t* __restrict__ part) {
  const int64_t total = (int64_t)(n + nnz);
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= units;
       u += (uint64_t)gridDim.x * blockDim.x) {
    int64_t d = (int64_t)(u * grain);
    if (d > total) d = total;
    const int64_t rows = merge_path_rows(offsets, (int64_t)n, (int64_t)nnz, d);
    part[2 * u] = rows;
    part[2 * u + 1] = d - rows;
  }
}

// edge pass (checkwalk.cuh): uncovered entries, in the rows of unmatched vertices
__global__ void validate_edges_kernel(uint64_t n, uint64_t nnz, const int64_t* __restrict__ offsets,
                                      const uint32_t* __restrict__ nbrs,
                                      const uint32_t* __restrict__ mate,
                                      const int64_t* __restrict__ part, uint64_t units,
                                      unsigned long long* __restrict__ c) {
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long unc = 0, first = ~0ull;
  for (uint64_t u = warp; u < units; u += nwarps) {
    const int64_t e0 = part[2 * u + 1], e1 = part[2 * u + 3];
    if (e0 < e1) check_unit(offsets, nbrs, n, nnz, mate, part[2 * u], e0, e1, lane, unc, first);
  }
  unc = warp_sum64(unc);
  first = warp_min64(first);
  if (lane == 0) {
    if (unc) atomicAdd(c + C_UNCOVERED, unc);
    if (first != ~0ull) atomicMin(c + C_FIRST_UNCOVERED, first);
  }
}

// edge pass over an edge list: edge i = (x, y), x != y, both ids < n, is
// uncovered when both endpoints are unmatched; mate[x] == y marks found[x] and
// mate[y] == x marks found[y] (the listed edge is the output edge of x / y)
__global__ void validate_coo_edges_kernel(uint64_t n, uint64_t m, const uint32_t* __restrict__ src,
                                          const uint32_t* __restrict__ dst,
                                          const uint32_t* __restrict__ mate,
                                          unsigned char* __restrict__ found,
                                          unsigned long long* __restrict__ c) {
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long unc = 0, first = ~0ull;
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < m; i0 += stride) {
    const uint64_t i = i0 + threadIdx.x;
    if (i < m) {
      const uint32_t x = __ldg(src + i), y = __ldg(dst + i);
      if (x != y && x < n && y < n) {
        const uint32_t mx = __ldg(mate + x), my = __ldg(mate + y);
        if (mx == kNone && my == kNone) {
          ++unc;
          if (i < first) first = i;
        }
        if (mx == y) found[x] = 1;
        if (my == x) found[y] = 1;
      }
    }
  }
  unc = warp_sum64(unc);
  first = warp_min64(first);
  if (lane == 0) {
    if (unc) atomicAdd(c + C_UNCOVERED, unc);
    if (first != ~0ull) atomicMin(c + C_FIRST_UNCOVERED, first);
  }
}

// existence pass (checkwalk.cuh): each named partner must share an edge with
// its vertex; one warp per 32 consecutive vertices
__global__ void validate_exist_kernel(uint64_t n, const int64_t* __restrict__ offsets,
                                      const uint32_t* __restrict__ nbrs,
                                      const uint32_t* __restrict__ mate,
                                      unsigned long long* __restrict__ c) {
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long nonedge = 0, first = ~0ull;
  for (uint64_t v0 = warp * 32; v0 < n; v0 += nwarps * 32)
    check_pairs32(offsets, nbrs, n, mate, v0, lane, nonedge, first);
  if (lane == 0) {
    if (nonedge) atomicAdd(c + C_NONEDGE, nonedge);
    if (first != ~0ull) atomicMin(c + C_FIRST_BAD, first);
  }
}

// vertex pass: range / symmetry of each named partner; with `found` (edge
// lists: the edge pass marks every vertex whose partner edge it met) also its
// existence -- a CSR's existence pass is validate_exist_kernel
__global__ void validate_vertex_kernel(uint64_t n, const uint32_t* __restrict__ mate,
                                       const unsigned char* __restrict__ found,
                                       unsigned long long* __restrict__ c) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x; v0 < n; v0 += stride) {
    const uint64_t v = v0 + threadIdx.x;
    uint32_t matched = 0, pair = 0, range = 0, asym = 0, nonedge = 0;
    bool bad = false;
    if (v < n) {
      const uint32_t m = mate[v];
      if (m != kNone) {
        if (m >= n || m == v) {
          range = 1;
          bad = true;
        } else {
          matched = 1;
          if (mate[m] != (uint32_t)v) {
            asym = 1;
            bad = true;
          } else if (v < m) {
            pair = 1;
          }
          if (found && !found[v] && !found[m]) {  // the edge may be listed either way
            nonedge = 1;
            bad = true;
          }
        }
      }
    }
    warp_add(c + C_MATCHED, matched);
    warp_add(c + C_PAIRS, pair);
    warp_add(c + C_RANGE, range);
    warp_add(c + C_ASYM, asym);
    warp_add(c + C_NONEDGE, nonedge);
    const uint32_t first_bad = __reduce_min_sync(kFull, bad ? (uint32_t)v : kNone);
    if ((threadIdx.x & 31) == 0 && first_bad != kNone) atomicMin(c + C_FIRST_BAD, (unsigned long long)first_bad);
  }
}

__global__ void validate_pairs_kernel(uint64_t n, const uint32_t* __restrict__ mate,
                                      const uint32_t* __restrict__ pairs, uint64_t count,
                                      uint32_t* __restrict__ seen, unsigned long long* __restrict__ c) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j0 = (uint64_t)blockIdx.x * blockDim.x; j0 < count; j0 += stride) {
    const uint64_t j = j0 + threadIdx.x;
    uint32_t bad = 0;
    if (j < count) {
      const uint32_t a = pairs[2 * j], b = pairs[2 * j + 1];
      const bool valid = a < b && b < n && mate[a] == b && mate[b] == a;
      if (!valid) {
        bad = 1;
      } else {
        const uint32_t bit = 1u << (a & 31u);
        if (atomicOr(seen + (a >> 5), bit) & bit) bad = 1;  // a repeat of a valid pair
      }
    }
    warp_add(c + C_PAIRS_BAD, bad);
  }
}

// ---- ordered compaction of (u, mate[u]), u < mate[u] ----
constexpr int kCompactThreads = 256;
constexpr int kPerThread = (int)(kCompactTile / kCompactThreads);  // 16

__device__ __forceinline__ bool takes(const uint32_t* mate, uint64_t n, uint64_t u) {
  if (u >= n) return false;
  const uint32_t m = mate[u];
  return m != kNone && m < n && u < m;
}

__global__ void compact_count_kernel(uint64_t n, const uint32_t* __restrict__ mate,
                                     uint64_t* __restrict__ tile_counts) {
  const uint64_t base = (uint64_t)blockIdx.x * kCompactTile + (uint64_t)threadIdx.x * kPerThread;
  uint32_t cnt = 0;
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) cnt += takes(mate, n, base + i);
  __shared__ uint32_t warp_sums[kCompactThreads / 32];
  const uint32_t ws = __reduce_add_sync(kFull, cnt);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < kCompactThreads / 32; ++w) t += warp_sums[w];
    tile_counts[blockIdx.x] = t;
  }
}

// exclusive scan of the tile counts in place (one block); total -> *count
__global__ void compact_scan_kernel(uint64_t tiles, uint64_t* __restrict__ tile_counts,
                                    uint64_t* __restrict__ count) {
  __shared__ uint64_t carry_s;
  __shared__ uint64_t warp_tot[32];
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint64_t b = 0; b < tiles; b += blockDim.x) {
    const uint64_t i = b + threadIdx.x;
    const uint64_t v = i < tiles ? tile_counts[i] : 0;
    uint64_t x = v;  // inclusive warp scan
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t y = __shfl_up_sync(kFull, x, d);
      if ((int)lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint64_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(kFull, t, d);
        if ((int)lane >= d) t += y;
      }
      if (lane < nw) warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const uint64_t before = carry_s + (wid ? warp_tot[wid - 1] : 0) + x - v;
    if (i < tiles) tile_counts[i] = before;
    __syncthreads();
    if (threadIdx.x == 0) carry_s += warp_tot[nw - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0 && count) *count = carry_s;
}

__global__ void compact_scatter_kernel(uint64_t n, const uint32_t* __restrict__ mate,
                                       const uint64_t* __restrict__ tile_offsets,
                                       uint32_t* __restrict__ pairs, uint64_t cap) {
  const uint64_t base = (uint64_t)blockIdx.x * kCompactTile + (uint64_t)threadIdx.x * kPerThread;
  uint32_t flags = 0, cnt = 0;
#pragma unroll
  for (int i = 0; i < kPerThread; ++i)
    if (takes(mate, n, base + i)) {
      flags |= 1u << i;
      ++cnt;
    }
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, d);
    if ((int)lane >= d) x += y;
  }
  __shared__ uint32_t warp_tot[kCompactThreads / 32];
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  uint32_t wbefore = 0;
  for (unsigned w = 0; w < wid; ++w) wbefore += warp_tot[w];
  uint64_t pos = tile_offsets[blockIdx.x] + wbefore + x - cnt;
#pragma unroll
  for (int i = 0; i < kPerThread; ++i)
    if (flags >> i & 1u) {
      if (pos < cap) {
        pairs[2 * pos] = (uint32_t)(base + i);
        pairs[2 * pos + 1] = mate[base + i];
      }
      ++pos;
    }
}

}  // namespace

cudaError_t launch_csr_check(uint64_t n, uint64_t nnz, const int64_t* offsets,
                             const uint32_t* nbrs, unsigned long long* bad, int grid,
                             cudaStream_t s) {
  zero_u64_kernel<<<1, 32, 0, s>>>(bad, 1, 0ull);
  csr_check_kernel<<<grid, 256, 0, s>>>(n, nnz, offsets, nbrs, bad);
  return cudaGetLastError();
}

cudaError_t launch_validate(uint64_t n, uint64_t nnz, const int64_t* offsets, const uint32_t* nbrs,
                            const uint32_t* mate, const uint32_t* pairs, uint64_t count,
                            const CheckScratch& cs, int grid, cudaStream_t s) {
  zero_u64_kernel<<<1, 32, 0, s>>>(cs.counters, C_FIRST_BAD, 0ull);
  zero_u64_kernel<<<1, 32, 0, s>>>(cs.counters + C_FIRST_BAD, 2, ~0ull);
  if (pairs && count) zero_u32_kernel<<<grid, 256, 0, s>>>(cs.seen_bits, (n + 31) / 32);
  if (n) {
    const uint64_t units = (n + nnz + kCheckGrain - 1) / kCheckGrain;
    check_partition_kernel<<<grid, 256, 0, s>>>(n, nnz, offsets, kCheckGrain, units, cs.part);
    if (nnz) validate_edges_kernel<<<grid, 256, 0, s>>>(n, nnz, offsets, nbrs, mate, cs.part, units, cs.counters);
    validate_exist_kernel<<<grid, 256, 0, s>>>(n, offsets, nbrs, mate, cs.counters);
    validate_vertex_kernel<<<grid, 256, 0, s>>>(n, mate, nullptr, cs.counters);
  }
  if (pairs && count) validate_pairs_kernel<<<grid, 256, 0, s>>>(n, mate, pairs, count, cs.seen_bits, cs.counters);
  return cudaGetLastError();
}

cudaError_t launch_coo_check(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                             unsigned long long* bad, int grid, cudaStream_t s) {
  zero_u64_kernel<<<1, 32, 0, s>>>(bad, 1, 0ull);
  if (m) coo_check_kernel<<<grid, 256, 0, s>>>(n, m, src, dst, bad);
  return cudaGetLastError();
}

cudaError_t launch_validate_coo(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                                const uint32_t* mate, const uint32_t* pairs, uint64_t count,
                                const CheckScratch& cs, int grid, cudaStream_t s) {
  zero_u64_kernel<<<1, 32, 0, s>>>(cs.counters, C_FIRST_BAD, 0ull);
  zero_u64_kernel<<<1, 32, 0, s>>>(cs.counters + C_FIRST_BAD, 2, ~0ull);
  if (pairs && count) zero_u32_kernel<<<grid, 256, 0, s>>>(cs.seen_bits, (n + 31) / 32);
  if (n) {
    zero_u32_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<uint32_t*>(cs.found), (n + 3) / 4);
    if (m) validate_coo_edges_kernel<<<grid, 256, 0, s>>>(n, m, src, dst, mate, cs.found, cs.counters);
    validate_vertex_kernel<<<grid, 256, 0, s>>>(n, mate, cs.found, cs.counters);
  }
  if (pairs && count) validate_pairs_kernel<<<grid, 256, 0, s>>>(n, mate, pairs, count, cs.seen_bits, cs.counters);
  return cudaGetLastError();
}

namespace {

// Census of a state array: out[0..3] = ACC, RSVD, MCHD, other field values.
__global__ void census_kernel(const uint32_t* __restrict__ state, uint64_t n, int bits,
                              unsigned long long* __restrict__ out) {
  unsigned long long c[4] = {0, 0, 0, 0};
  const uint64_t per = bits == 32 ? 1 : 32u / (uint32_t)bits;
  const uint32_t mask = bits == 32 ? 0u : (1u << bits) - 1u;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t w = state[v / per];
    int k;
    if (bits == 32) {
      k = w == kWAcc ? 0 : (w == kWRsvd ? 1 : 2);
    } else {
      const uint32_t f = (w >> ((v % per) * (uint32_t)bits)) & mask;
      k = f == kAcc ? 0 : f == kRsvd ? 1 : f == kMchd ? 2 : 3;
    }
    ++c[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned long long t = warp_sum64(c[k]);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(out + k, t);
  }
}

}  // namespace

cudaError_t launch_census(const uint32_t* state, uint64_t n, int bits, unsigned long long* out,
                          int grid, cudaStream_t s) {
  zero_u64_kernel<<<1, 32, 0, s>>>(out, 4, 0ull);
  if (n) census_kernel<<<grid, 256, 0, s>>>(state, n, bits, out);
  return cudaGetLastError();
}

cudaError_t launch_compact(uint64_t n, const uint32_t* mate, uint32_t* pairs, uint64_t cap,
                           uint64_t* count, const CheckScratch& cs, cudaStream_t s) {
  const uint64_t tiles = (n + kCompactTile - 1) / kCompactTile;
  if (tiles > cs.block_cap) return cudaErrorInvalidValue;
  if (tiles == 0) {
    if (count) zero_u64_kernel<<<1, 32, 0, s>>>(reinterpret_cast<unsigned long long*>(count), 1, 0ull);
    return cudaGetLastError();
  }
  compact_count_kernel<<<(unsigned)tiles, kCompactThreads, 0, s>>>(n, mate, cs.block_counts);
  compact_scan_kernel<<<1, 1024, 0, s>>>(tiles, cs.block_counts, count);
  if (pairs && cap)
    compact_scatter_kernel<<<(unsigned)tiles, kCompactThreads, 0, s>>>(n, mate, cs.block_counts, pairs, cap);
  return cudaGetLastError();
}

}  // namespace skp
