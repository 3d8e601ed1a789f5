// coo.cu -- Skipper over a list of edges in coordinate form on sm_103a.
//
// Section V-C: Skipper does not depend on the input format; it can read the
// edges as a list (src[i], dst[i]), each undirected edge once, in any order and
// either direction, with no symmetrisation.  Algorithm 1 is then run for every
// listed edge (lines 5-18 with the list in place of the CSR walk).  There is no
// row to leave, so every edge is read; the work per edge is one 8-byte read of
// its endpoints and the two line-10 state reads.
//
// coo_prepare_kernel: Algorithm 1 lines 3-4 (every vertex ACC, mate unmatched).
// coo_sweep_kernel: persistent warps take units of `grain` edges from a global
//   counter and walk them 128 edges at a time: one 128-bit load of src and one
//   of dst per lane (4 edges a lane), the eight state reads issued together,
//   then the candidates (both endpoints unmatched) are tried in rounds of one
//   edge per lane.  Lanes whose edges reserve the same vertex u first (u = the
//   lower endpoint, Alg. 1 lines 8-9) elect one leader per round; when the
//   leader leaves u matched the others drop their edge without an attempt, so a
//   run of edges sharing one vertex (a list in CSR order) costs one round.
// coo_serial_kernel: one thread, edges in list order -- the sequential greedy
//   order, identical to SGMM over the list.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "walk.cuh"

namespace skp {

namespace {

__global__ void coo_prepare_kernel(CooParams C, int bits) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const SweepParams& P = C.P;
  const uint64_t n = P.n;
  const bool poison = P.poison != 0;
  const uint64_t pv = poison ? P.poison - 1 : 0;
  if (bits == 32) {
    for (uint64_t i = tid; i < n; i += nthreads) P.state[i] = (poison && i == pv) ? kWRsvd : kWAcc;
  } else {
    const uint64_t per = 32u / (uint32_t)bits;
    const uint64_t words = packed_words(n, bits);
    for (uint64_t i = tid; i < words; i += nthreads)
      P.state[i] = (poison && i == pv / per) ? (kRsvd << ((pv % per) * (uint64_t)bits)) : 0u;
    for (uint64_t i = tid; i < n; i += nthreads) P.mate[i] = kNone;
  }
  if (P.stats && tid < kStCount) P.stats[tid] = 0ull;
  if (tid == 0) {
    *P.work = 0ull;
    *P.err = 0u;
  }
}

// The 4 edges of one lane: entries [i0, i0 + 4) of the list, clipped to e_hi.
template <bool kVec>
__device__ __forceinline__ void load_edges(const CooParams& C, uint64_t i0, uint64_t e_hi,
                                           uint64_t pol, uint32_t (&x)[4], uint32_t (&y)[4]) {
  if (kVec && i0 + 4 <= e_hi) {
    const uint4 a = ld_stream_v4(C.src + i0, pol);
    const uint4 b = ld_stream_v4(C.dst + i0, pol);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    y[0] = b.x; y[1] = b.y; y[2] = b.z; y[3] = b.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool in = i0 + j < e_hi;
      x[j] = in ? ld_stream(C.src + i0 + j, pol) : 0u;
      y[j] = in ? ld_stream(C.dst + i0 + j, pol) : 0u;
    }
  }
}

template <class S, bool kStats, bool kVec>
__global__ void __launch_bounds__(512, 3) coo_sweep_kernel(CooParams C) {
  const unsigned lane = threadIdx.x & 31u;
  const SweepParams& P = C.P;
  const S s(P);
  const uint64_t pol = policy_evict_first();
  const uint32_t n32 = (uint32_t)P.n;
  for (;;) {
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(P.work, 1ull);
    w = __shfl_sync(kFull, w, 0);
    if (w >= C.units) return;
    const uint64_t e_lo = w * C.grain;
    const uint64_t e_hi = e_lo + C.grain < C.m ? e_lo + C.grain : C.m;
    for (uint64_t t = e_lo; t < e_hi; t += 128) {
      const uint64_t i0 = t + 4 * lane;
      uint32_t x[4], y[4];
      load_edges<kVec>(C, i0, e_hi, pol, x, y);
      if (kStats && lane == 0) {
        atomicAdd(P.stats + kStChunks, 1ull);
        atomicAdd(P.stats + kStEntries, (unsigned long long)(e_hi - t < 128 ? e_hi - t : 128));
      }
      // line 10 for every listed edge: the four src states first, then the dst
      // states of the edges whose src is not matched (most edges end here)
      bool live[4];
      uint32_t rx[4], ry[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        live[j] = i0 + j < e_hi && x[j] != y[j];  // lines 6-7: loops are skipped
        if (live[j] && (x[j] >= n32 || y[j] >= n32)) {
          atomicOr(P.err, kErrBadId);
          live[j] = false;
        }
        rx[j] = live[j] ? s.peek(x[j]) : 0u;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        live[j] = live[j] && !S::matched(rx[j], x[j]);
        ry[j] = live[j] ? s.peek(y[j]) : 0u;
      }
      uint32_t cand = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (live[j] && !S::matched(ry[j], y[j])) cand |= 1u << j;

      // rounds: one candidate per lane, one leader per reserved-first vertex u
      for (bool first = true;; first = false) {
        bool have = cand != 0u;
        if (!__any_sync(kFull, have)) break;
        const int j = have ? __ffs(cand) - 1 : 0;
        const uint32_t xj = pick4(x, j), yj = pick4(y, j);
        const bool x_low = xj < yj;
        const uint32_t u = x_low ? xj : yj, v = x_low ? yj : xj;
        uint32_t ru = 0, rv = 0;
        if (have) {
          if (first) {
            const uint32_t wx = pick4(rx, j), wy = pick4(ry, j);
            ru = x_low ? wx : wy;
            rv = x_low ? wy : wx;
          } else {  // an earlier round may have matched either endpoint: read line 10 again
            ru = s.peek(u);
            rv = s.peek(v);
            if (S::matched(ru, u) || S::matched(rv, v)) {
              cand &= ~(1u << j);
              have = false;
            }
          }
        }
        const uint32_t key = have ? u : kNone;
        const unsigned peers = __match_any_sync(kFull, key);
        const int leader = __ffs(peers) - 1;
        bool u_done = false;
        if (have && (int)lane == leader) {
          cand &= ~(1u << j);
          u_done = resolve_edge<S, kStats>(s, u, v, ru, rv, P);
        }
        u_done = __shfl_sync(kFull, u_done, leader);
        if (have && u_done) cand &= ~(1u << j);  // u is matched: the peers' edges are covered
      }
    }
    if ((w & 15) == 0) {  // stop handing out work once an error is recorded
      uint32_t e = 0;
      if (lane == 0) e = ld_relaxed(P.err);
      if (__shfl_sync(kFull, e, 0) & kErrTimeout) return;
    }
  }
}

template <class S>
__global__ void coo_serial_kernel(CooParams C) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const SweepParams& P = C.P;
  const S s(P);
  for (uint64_t i = 0; i < C.m; ++i) {
    const uint32_t x = C.src[i], y = C.dst[i];
    if (x >= P.n || y >= P.n) {
      atomicOr(P.err, kErrBadId);
      continue;
    }
    if (x == y) continue;
    resolve_edge(s, x, y, s.raw(x), s.raw(y), P);
    if (ld_relaxed(P.err) & kErrTimeout) return;
  }
}

}  // namespace

#define SKP_COO_STATE(bits, F) \
  ((bits) == 32 ? F(WordState) : (bits) == 2 ? F(TwoBitState) : F(ByteState))

int coo_blocks_per_sm(int bits, int block_threads) {
  int b = 0;
#define OCC(S) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, coo_sweep_kernel<S, false, true>, block_threads, 0)
  cudaError_t e = SKP_COO_STATE(bits, OCC);
#undef OCC
  if (e != cudaSuccess || b < 1) return 1;
  return b;
}

cudaError_t launch_coo_prepare(const CooParams& C, int bits, int grid, cudaStream_t s) {
  coo_prepare_kernel<<<grid, 256, 0, s>>>(C, bits);
  return cudaGetLastError();
}

cudaError_t launch_coo_sweep(const CooParams& C, int bits, int grid, int block, cudaStream_t s) {
  if (block > 512 || block < 32 || block % 32) return cudaErrorInvalidValue;
  if (C.units == 0) return cudaSuccess;
  const bool vec = C.vec != 0;
#define L(S)                                                                             \
  (C.P.stats ? (vec ? (coo_sweep_kernel<S, true, true><<<grid, block, 0, s>>>(C), 0)     \
                    : (coo_sweep_kernel<S, true, false><<<grid, block, 0, s>>>(C), 0))   \
             : (vec ? (coo_sweep_kernel<S, false, true><<<grid, block, 0, s>>>(C), 0)    \
                    : (coo_sweep_kernel<S, false, false><<<grid, block, 0, s>>>(C), 0)))
  SKP_COO_STATE(bits, L);
#undef L
  return cudaGetLastError();
}

cudaError_t launch_coo_serial(const CooParams& C, int bits, cudaStream_t s) {
#define L(S) (coo_serial_kernel<S><<<1, 1, 0, s>>>(C), 0)
  SKP_COO_STATE(bits, L);
#undef L
  return cudaGetLastError();
}

}  // namespace skp
