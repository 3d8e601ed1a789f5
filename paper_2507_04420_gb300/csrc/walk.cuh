// walk.cuh -- the per-warp walk of Skipper's single pass (Algorithm 1) over
// one merge-path work unit, shared by the single-graph sweep (sweep.cu) and
// the multi-graph sweep (multi.cu).  Every function here takes the graph it
// works on through a SweepParams view, so one unit of any graph is walked the
// same way.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "state.cuh"

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

// Four neighbour ids from entry e0 on (one aligned 128-bit load when all four
// exist, else the ones below nnz).
__device__ __forceinline__ void load_quad(const SweepParams& P, int64_t e0, uint64_t pol,
                                          uint32_t (&y)[4]) {
  if (e0 + 4 <= (int64_t)P.nnz) {
    const uint4 q = ld_stream_v4(P.nbrs + e0, pol);
    y[0] = q.x; y[1] = q.y; y[2] = q.z; y[3] = q.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (e0 + j < (int64_t)P.nnz) y[j] = ld_stream(P.nbrs + e0 + j, pol);
  }
}

// Shared-memory tile of one 32-row window (kTile instances, opt-in), filled
// by one bulk copy (TMA, cp.async.bulk with an mbarrier) while the warp still
// works on the window before it: the window's row ends (34 int64 from an even
// index, 272 bytes) and the state words of its rows (12 words from a multiple
// of 4, 48 bytes).  Both copies start 16-byte aligned (the host enables the
// instances only for 16-byte aligned arrays in device memory) and stay inside
// their arrays (n + 1 row ends, ceil(n / per word) state words); a window for
// which they would not is loaded directly.  The state words are a snapshot one
// window old: a row matched since then reads as unmatched, which costs an
// extra filter read, never a wrong result (MCHD is absorbing, and every
// transition is a CAS on the current word).  Every wait on the barrier is
// bounded.
struct alignas(16) WindowTile {
  int64_t ends[36];
  uint32_t st[16];
  unsigned long long bar;
  unsigned long long pad;
};
constexpr uint32_t kTileEnds = 34, kTileWords = 12;
constexpr uint32_t kTileBytes = kTileEnds * 8 + kTileWords * 4;
__shared__ WindowTile g_window_tiles[16];       // one per warp of a block of <= 512 threads

// the warp's tile barrier (one arrival per copy); once per warp before its first unit
__device__ __forceinline__ void init_window_tile(unsigned lane) {
  if (lane == 0) {
    mbar_init(&g_window_tiles[threadIdx.x >> 5].bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
}

// One work unit: entries [e_begin, e_end), the first of which lies in row >= row0.
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
//
// kTile: windows come from the warp's shared-memory tile (WindowTile above).
//
// kSel (selective id loads): a lane loads its quad only after the row search,
// and only when the quad holds an entry of a row not known matched.  The
// eager walk issues every load of the chunk first, so that its latency
// overlaps the search; the selective walk moves fewer bytes (on R-MAT, well
// under half the quads of a chunk are in rows not known matched), which pays
// where the bytes cross the host link.
template <class S, bool kStats = false, bool kSym = false, bool kSel = false, bool kTile = false>
__device__ __forceinline__ void sweep_unit(const S& s, const SweepParams& P, int64_t row0,
                                           const int64_t e_begin, const int64_t e_end,
                                           const unsigned lane, const uint64_t pol_stream,
                                           uint32_t* phase = nullptr) {
  const uint32_t n32 = (uint32_t)P.n;
  // Positions are entry indices relative to e_begin (a unit holds at most
  // 2^24 items, so 32 bits suffice).  Row ends are clamped to [0, ue]: a row
  // that ends before the unit reads as ending at 0, one that ends after it as
  // ending at ue, which changes no comparison the walk makes.
  const int ue = (int)(e_end - e_begin);
  const int align = (int)(e_begin & 3);     // base of a chunk: ((pos + align) & ~3) - align
  auto rel_end = [&](int64_t end) -> int {
    const int64_t d = end - e_begin;
    return d < 0 ? 0 : (d > (int64_t)ue ? ue : (int)d);
  };
  int64_t wbase = row0;
  int my_end;
  uint32_t my_st;
  unsigned mchd;
  int pos = 0;
  bool pending = false;                         // a copy of the next window's tile is in flight
  auto tile = [&]() { return &g_window_tiles[threadIdx.x >> 5]; };
  auto t_s = [&](int64_t w) { return (w + 1) & ~(int64_t)1; };
  auto t_sw = [&](int64_t w) { return (w / (int64_t)S::kPerWord) & ~(int64_t)3; };
  auto issue_next = [&](int64_t w) {
    if (!kTile) return;
    const int64_t sidx = t_s(w), sw = t_sw(w);
    // both copies stay inside their arrays: n + 1 row offsets, ceil(n / per word) state words
    if (sidx + (int64_t)kTileEnds > (int64_t)P.n + 1 ||
        sw + (int64_t)kTileWords > (int64_t)((P.n + S::kPerWord - 1) / S::kPerWord))
      return;
    if (lane == 0) {
      fence_proxy_async_smem();   // this warp's reads of the tile come before the copy's writes
      mbar_expect_tx(&tile()->bar, kTileBytes);
      bulk_to_smem(tile()->ends, P.offsets + sidx, kTileEnds * 8, &tile()->bar);
      bulk_to_smem(tile()->st, P.state + sw, kTileWords * 4, &tile()->bar);
    }
    pending = true;
  };
  // bounded wait for the copy in flight; false when it ran past the limit
  auto wait_tile = [&]() -> bool {
    for (uint32_t i = 0; i < (1u << 22); ++i)
      if (mbar_try_wait(&tile()->bar, *phase)) {
        *phase ^= 1u;
        pending = false;
        return true;
      }
    return false;
  };
  {
    const int64_t r = wbase + lane;
    const bool in = r < (int64_t)P.n;
    my_end = in ? rel_end(__ldg(P.offsets + r + 1)) : ue;
    my_st = in ? s.peek((uint32_t)r) : 0u;
    mchd = __ballot_sync(kFull, !in || S::matched(my_st, (uint32_t)r));  // rows past n hold no entries
    issue_next(wbase + 32);
  }
  while (pos < ue) {
    // rows of the window with entries at or after pos that are not known matched
    const unsigned open = __ballot_sync(kFull, my_end > pos) & ~mchd;
    if (open == 0u) {  // the window is exhausted: continue after its last row
      const int win_end = __shfl_sync(kFull, my_end, 31);
      if (win_end >= ue) break;
      if (win_end > pos) pos = win_end;
      wbase += 32;
      const int64_t r = wbase + lane;
      const bool in = r < (int64_t)P.n;
      bool from_tile = false;
      if (kTile && pending) {
        from_tile = wait_tile();
        if (!from_tile) {            // the copy did not land: stop, after a last bounded wait
          if (lane == 0) atomicOr(P.err, kErrTimeout);
          wait_tile();
          return;
        }
      }
      if (from_tile) {
        my_end = in ? rel_end(tile()->ends[wbase + 1 + lane - t_s(wbase)]) : ue;
        my_st = in ? tile()->st[(r / (int64_t)S::kPerWord) - t_sw(wbase)] : 0u;
        __syncwarp();
      } else {
        my_end = in ? rel_end(__ldg(P.offsets + r + 1)) : ue;
        my_st = in ? s.peek((uint32_t)r) : 0u;
      }
      mchd = __ballot_sync(kFull, !in || S::matched(my_st, (uint32_t)r));
      issue_next(wbase + 32);
      if (kStats && lane == 0) atomicAdd(P.stats + kStWindows, 1ull);
      continue;
    }
    const int k1 = __ffs(open) - 1;
    if (k1 > 0) {  // row k1 starts where row k1-1 ends
      const int st = __shfl_sync(kFull, my_end, k1 - 1);
      if (st > pos) pos = st;
    }
    if (pos >= ue) break;
    const int win_end = __shfl_sync(kFull, my_end, 31);
    const int base = ((pos + align) & ~3) - align;
    int cend = base + 128;
    if (cend > ue) cend = ue;
    if (cend > win_end) cend = win_end;
    // chunk-relative coordinates: entry base+p, p in [lo_r, hi_r)
    const int lo_r = pos - base;
    const int hi_r = cend - base;
    if (kStats && lane == 0) {
      atomicAdd(P.stats + kStChunks, 1ull);
      atomicAdd(P.stats + kStEntries, (unsigned long long)(hi_r - lo_r));
    }
    int rel = my_end - base;
    rel = rel < 0 ? -1 : (rel > 129 ? 129 : rel);

    // neighbour ids (one aligned 128-bit load per lane) and, in parallel, a
    // fresh read of the head row's state
    const int p0 = 4 * (int)lane;
    const int64_t e0 = e_begin + base + p0;
    uint32_t y[4] = {0u, 0u, 0u, 0u};
    if (!kSel && p0 < hi_r) load_quad(P, e0, pol_stream, y);
    const uint32_t wb32 = (uint32_t)wbase;
    const uint32_t x1 = wb32 + (uint32_t)k1;
    uint32_t head = 0;
    if (lane == 0) head = s.peek(x1);  // consumed after the row search, so both loads overlap it

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
    head = __shfl_sync(kFull, head, 0);
    if (S::matched(head, x1)) mchd |= 1u << k1;
    if (lane == (unsigned)k1) my_st = head;
    uint32_t xs[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) xs[j] = wb32 + (uint32_t)k[j];
    if (kSel || kStats) {
      // does this lane's quad hold an entry of a row not known matched?
      bool open_quad = false;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int p = p0 + j;
        open_quad |= p >= lo_r && p < hi_r && !(mchd >> (k[j] & 31) & 1u);
      }
      if (kSel && open_quad) load_quad(P, e0, pol_stream, y);
      if (kStats) {
        const unsigned issued = __ballot_sync(kFull, p0 < hi_r);
        const unsigned wanted = __ballot_sync(kFull, open_quad);
        if (lane == 0) {
          atomicAdd(P.stats + kStIdLoads, (unsigned long long)__popc(issued));
          atomicAdd(P.stats + kStIdLoadsOpen, (unsigned long long)__popc(wanted));
        }
      }
    }

    // filter (the line-10 read): candidates have both endpoints unmatched.  A
    // row whose snapshot word reads MCHD has its bit in mchd (set when the
    // window or the head word was read), so the row test is the mask alone.
    // Loops are skipped (lines 6-7); on a symmetric CSR so is every (x, y) with
    // y < x, which row y holds as (y, x) (each edge tested once).
    bool want[4];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = p0 + j;
      want[j] = p >= lo_r && p < hi_r && !(mchd >> (k[j] & 31) & 1u) &&
                (kSym ? y[j] > xs[j] : y[j] != xs[j]);
      bad |= want[j] && y[j] >= n32;
      want[j] = want[j] && y[j] < n32;
    }
    if (__any_sync(kFull, bad) && bad) atomicOr(P.err, kErrBadId);
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
      const uint32_t rxj = __shfl_sync(kFull, my_st, (key - wb32) & 31);
      const unsigned peers = __match_any_sync(kFull, key);
      const int leader = __ffs(peers) - 1;
      unsigned done = 0u;
      if (have && (int)lane == leader) {
        cand &= ~(1u << j);
        if (resolve_edge<S, kStats>(s, key, pick4(y, j), rxj, pick4(ry, j), P))
          done = 1u << (key - wb32);
      }
      done = __reduce_or_sync(kFull, done);  // rows that are now matched
      mchd |= done;
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
        if (done >> (k[jj] & 31) & 1u) cand &= ~(1u << jj);
    }
    pos = cend;
  }
  if (kTile && pending && !wait_tile()) {   // the tile is reused by the next unit
    if (lane == 0) atomicOr(P.err, kErrTimeout);
    wait_tile();
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

}  // namespace
}  // namespace skp
