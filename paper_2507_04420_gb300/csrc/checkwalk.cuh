// checkwalk.cuh -- the exact checker's two graph passes (Section II-B: every
// graph edge touches an output edge; each output edge is a graph edge), shared
// by the single-graph and multi-graph checkers.
//
// Edge pass (check_unit), over one merge-path unit: an entry (x, y), x != y,
// is uncovered when mate[x] and mate[y] are both unmatched -- so only the rows
// of unmatched vertices can hold one.  The walk keeps 32-row windows (row ends
// and mates in one step, like the sweep) and leaves every row whose mate is
// set; the remaining entries are read 128 at a time.
//
// Existence pass (check_pairs32), over 32 consecutive vertices: a vertex v
// naming a partner m in range must share an edge with it, stored in row v or
// in row m (the CSR may hold an edge for one endpoint only).  The warp
// searches the shorter of the two rows first and stops at the first hit; a
// symmetric pair is searched once, by its lower endpoint, and counts for
// both.  Counting rules are those of the host checker.
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
                                           int64_t row0, int64_t pos, const int64_t e_end,
                                           const unsigned lane, unsigned long long& unc,
                                           unsigned long long& first_unc) {
  int64_t wbase = row0;
  int64_t my_end = 0;
  uint32_t my_mate = kNone;
  unsigned busy = 0;  // rows of the window whose mate is set: none of their entries is uncovered
  bool need = true;
  while (pos < e_end) {
    if (need) {
      const int64_t r = wbase + lane;
      const bool in = r < (int64_t)n;
      my_end = in ? __ldg(offsets + r + 1) : INT64_MAX;
      my_mate = in ? __ldg(mate + r) : kNone;
      busy = __ballot_sync(kFull, !in || my_mate != kNone);
      need = false;
    }
    const unsigned open = __ballot_sync(kFull, my_end > pos) & ~busy;
    const int64_t win_end = __shfl_sync(kFull, my_end, 31);
    if (open == 0u) {  // nothing left to check in this window
      if (win_end >= e_end) return;
      if (win_end > pos) pos = win_end;
      wbase += 32;
      need = true;
      continue;
    }
    const int k1 = __ffs(open) - 1;
    if (k1 > 0) {  // row k1 starts where row k1-1 ends
      const int64_t st = __shfl_sync(kFull, my_end, k1 - 1);
      if (st > pos) pos = st;
    }
    if (pos >= e_end) return;
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
      const int p = p0 + j;
      if (p < lo_r || p >= hi_r || (busy >> (k & 31) & 1u)) continue;
      const uint32_t x = (uint32_t)(wbase + k);
      if (y[j] == x || y[j] >= n) continue;
      if (__ldg(mate + y[j]) == kNone) {
        ++unc;
        const unsigned long long e = (unsigned long long)(e0 + j);
        if (e < first_unc) first_unc = e;
      }
    }
    pos = cend;
  }
}

// Does row r hold the id t?  The whole warp reads the row, 32 entries a step.
__device__ __forceinline__ bool warp_row_has(const int64_t* __restrict__ offsets,
                                             const uint32_t* __restrict__ nbrs, uint32_t r,
                                             uint32_t t, unsigned lane) {
  const int64_t s = __ldg(offsets + r), e = __ldg(offsets + r + 1);
  for (int64_t i = s; i < e; i += 32) {
    const int64_t k = i + lane;
    if (__any_sync(kFull, k < e && __ldg(nbrs + k) == t)) return true;
  }
  return false;
}

// Existence pass for vertices [v0, v0 + 32) of one graph (lane i: vertex v0 + i).
// Adds to `nonedge` (lane 0) the vertices whose named partner shares no edge
// with them, and lowers `first_bad` to the smallest of them.
__device__ __forceinline__ void check_pairs32(const int64_t* __restrict__ offsets,
                                              const uint32_t* __restrict__ nbrs, uint64_t n,
                                              const uint32_t* __restrict__ mate, uint64_t v0,
                                              unsigned lane, unsigned long long& nonedge,
                                              unsigned long long& first_bad) {
  const uint64_t v = v0 + lane;
  const uint32_t m = v < n ? __ldg(mate + v) : kNone;
  const bool valid = m != kNone && m < n && m != v;
  const bool sym = valid && __ldg(mate + m) == (uint32_t)v;
  unsigned todo = __ballot_sync(kFull, valid && !(sym && m < v));
  while (todo) {
    const int j = __ffs(todo) - 1;
    todo &= todo - 1;
    const uint32_t vj = (uint32_t)__shfl_sync(kFull, (unsigned)v, j);
    const uint32_t mj = __shfl_sync(kFull, m, j);
    const bool sj = __shfl_sync(kFull, sym ? 1u : 0u, j) != 0u;
    const int64_t dv = __ldg(offsets + vj + 1) - __ldg(offsets + vj);
    const int64_t dm = __ldg(offsets + mj + 1) - __ldg(offsets + mj);
    const bool v_first = dv <= dm;  // the shorter row first
    bool hit = warp_row_has(offsets, nbrs, v_first ? vj : mj, v_first ? mj : vj, lane);
    if (!hit) hit = warp_row_has(offsets, nbrs, v_first ? mj : vj, v_first ? vj : mj, lane);
    if (!hit && lane == 0) {
      nonedge += sj ? 2 : 1;
      if (vj < first_bad) first_bad = vj;  // a symmetric pair is searched by its lower end
    }
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
