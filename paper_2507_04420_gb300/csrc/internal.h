// internal.h -- launchers shared by the translation units of libskipper.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "state.cuh"

namespace skp {

// sweep.cu (bits: 2, 8 or 32 -- the state layout, see state.cuh)
int sweep_blocks_per_sm(int bits, int block_threads);
cudaError_t launch_prepare(const SweepParams& P, int bits, int grid, cudaStream_t s,
                           uint64_t* graph_pairs_zero, uint64_t num_graphs);
cudaError_t launch_sweep(const SweepParams& P, int bits, int grid, int block, cudaStream_t s);
cudaError_t launch_serial(const SweepParams& P, int bits, cudaStream_t s);
cudaError_t launch_serial_batched(const SweepParams& P, int bits, cudaStream_t s);
void get_batched_kernels(int bits, bool serial, bool sym, const void** prepare, const void** sweep,
                         const void** pairs);
cudaError_t launch_graph_pairs(const uint32_t* mate, const int64_t* vbase, uint64_t num_graphs,
                               uint64_t n, uint64_t* graph_pairs, int grid, cudaStream_t s);

// coo.cu: Skipper over an edge list (src[i], dst[i]) in coordinate form
struct CooParams {
  SweepParams P;        // n, state, mate, work, err, spin_limit, poison, stats (CSR fields unused)
  const uint32_t* src;  // m endpoint ids
  const uint32_t* dst;  // m endpoint ids
  uint64_t m;           // listed edges
  uint64_t units;       // ceil(m / grain)
  uint32_t grain;       // edges per work unit, a multiple of 128
  uint32_t vec;         // 1 when src and dst are 16-byte aligned (128-bit loads)
};
int coo_blocks_per_sm(int bits, int block_threads);
cudaError_t launch_coo_prepare(const CooParams& C, int bits, int grid, cudaStream_t s);
cudaError_t launch_coo_sweep(const CooParams& C, int bits, int grid, int block, cudaStream_t s);
cudaError_t launch_coo_serial(const CooParams& C, int bits, cudaStream_t s);

// api.cu: message returned by mm_last_error() on this thread
void set_error_message(const char* fmt, ...);

// check.cu
struct CheckScratch {
  unsigned long long* counters;  // mm_verdict-shaped device block (see check.cu)
  uint32_t* seen_bits;           // ceil(n/32) words
  uint64_t* block_counts;        // compaction: one count per tile of vertices
  uint64_t block_cap;
  unsigned char* found;          // edge-list checker: n bytes (+3), partner edge met in the list
  int64_t* part;                 // checker: merge-path table, (n+nnz)/kCheckGrain + 1 pairs
};
constexpr uint64_t kCheckGrain = 4096;  // rows + entries per checker work unit
cudaError_t launch_csr_check(uint64_t n, uint64_t nnz, const int64_t* offsets,
                             const uint32_t* nbrs, unsigned long long* bad, int grid,
                             cudaStream_t s);
cudaError_t launch_validate(uint64_t n, uint64_t nnz, const int64_t* offsets, const uint32_t* nbrs,
                            const uint32_t* mate, const uint32_t* pairs, uint64_t count,
                            const CheckScratch& cs, int grid, cudaStream_t s);
cudaError_t launch_coo_check(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                             unsigned long long* bad, int grid, cudaStream_t s);
cudaError_t launch_validate_coo(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                                const uint32_t* mate, const uint32_t* pairs, uint64_t count,
                                const CheckScratch& cs, int grid, cudaStream_t s);
cudaError_t launch_census(const uint32_t* state, uint64_t n, int bits, unsigned long long* out,
                          int grid, cudaStream_t s);
constexpr uint64_t kCompactTile = 4096;  // vertices per compaction tile
cudaError_t launch_compact(uint64_t n, const uint32_t* mate, uint32_t* pairs, uint64_t cap,
                           uint64_t* count, const CheckScratch& cs, cudaStream_t s);

}  // namespace skp
