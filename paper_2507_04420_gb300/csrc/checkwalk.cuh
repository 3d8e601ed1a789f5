// checkwalk.cuh -- the edge pass of the exact checker (Section II-B: every
// graph edge touches an output edge; each output edge is a graph edge), over
// one merge-path unit of a graph, shared by the single-graph and multi-graph
// checkers.
//
// Every stored entry (x, y), x != y, of the unit is read once (128 per warp
// step, one 128-bit load per lane, rows from a 32-row window like the sweep):
//   * mate[x] unmatched: the entry is uncovered when mate[y] is unmatched too;
//   * mate[x] == y: x's output edge is present in the graph (found[x] = 1).
// A vertex pass then needs no row scan: the output edge {v, m} exists when
// found[v] or found[m] is set (the edge may be stored for one endpoint only).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "state.cuh"

namespace skp {
namespace {

__device__ __forceinline__ int check_count_le(int rel, int p) {
  int c = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const int v = __shfl_sync(kFull, rel, c + step - 1);
    if (v <= p) c += step;
  }
  return c;
}

// Accumulates, per lane, the uncovered entries and the smallest such index.
__device__ __forceinline__ void check_unit(const int64_t* __restrict__ offsets,
                                           const uint32_t* __restrict__ nbrs, uint64_t n,
                                           uint64_t nnz, const uint32_t* __restrict__ mate,
                                           unsigned char* __restrict__ found, int64_t row0,
                                           int64_t pos, const int64_t e_end, const unsigned lane,
                                           unsigned long long& unc, unsigned long long& first_unc) {
  int64_t wbase = row0;
  int64_t my_end = 0;
  uint32_t my_mate = kNone;
  bool need = true;
  while (pos < e_end) {
    if (need) {
      const int64_t r = wbase + lane;
      const bool in = r < (int64_t)n;
      my_end = in ? __ldg(offsets + r + 1) : INT64_MAX;
      my_mate = in ? __ldg(mate + r) : kNone;
      need = false;
    }
    const int64_t win_end = __shfl_sync(kFull, my_end, 31);
    if (win_end <= pos) {  // every row of the window ends at or before pos
      wbase += 32;
      need = true;
      continue;
    }
    const int64_t base = pos & ~(int64_t)3;
    int64_t cend = base + 128;
    if (cend > e_end) cend = e_end;
    if (cend > win_end) cend = win_end;
    const int lo_r = (int)(pos - base), hi_r = (int)(cend - base);
    const int64_t rel64 = my_end - base;
    const int rel = rel64 < 0 ? -1 : (rel64 > 129 ? 129 : (int)rel64);
    const int p0 = 4 * (int)lane;
    const int64_t e0 = base + p0;
    uint32_t y[4] = {0u, 0u, 0u, 0u};
    if (p0 < hi_r) {
      if (e0 + 4 <= (int64_t)nnz) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(nbrs + e0));
        y[0] = q.x; y[1] = q.y; y[2] = q.z; y[3] = q.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (e0 + j < (int64_t)nnz) y[j] = __ldg(nbrs + e0 + j);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = check_count_le(rel, p0 + j);
      const uint32_t mx = __shfl_sync(kFull, my_mate, k & 31);
      const int p = p0 + j;
      if (p < lo_r || p >= hi_r) continue;
      const uint32_t x = (uint32_t)(wbase + k);
      if (y[j] == x || y[j] >= n) continue;
      if (mx == kNone) {
        if (__ldg(mate + y[j]) == kNone) {
          ++unc;
          const unsigned long long e = (unsigned long long)(e0 + j);
          if (e < first_unc) first_unc = e;
        }
      } else if (mx == y[j]) {
        found[x] = 1;
      }
    }
    pos = cend;
  }
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
  return v;
}

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(kFull, v, d);
    v = o < v ? o : v;
  }
  return v;
}

}  // namespace
}  // namespace skp
