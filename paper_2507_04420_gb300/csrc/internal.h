// internal.h -- launchers shared by the translation units of libskipper.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "state.cuh"

namespace skp {

// sweep.cu (bits: 2, 8 or 32 -- the state layout, see state.cuh)
// blocks of block_threads per SM that the default (lean = false) or the
// 32-register (lean = true) instance fits
int sweep_blocks_per_sm(int bits, int block_threads, bool lean);
// which instance a parallel CSR sweep uses: the 32-register one when the caller
// asks for more blocks per SM than the default fits, or by default when the
// state array takes at most half the L2 (it then stays there, and more warps
// hide more latency; a larger array's random sectors already load the memory)
bool sweep_lean(int bits, int block_threads, int blocks_per_sm, bool state_fits_l2);
cudaError_t launch_prepare(const SweepParams& P, int bits, int grid, cudaStream_t s,
                           uint64_t* graph_pairs_zero, uint64_t num_graphs);
cudaError_t launch_sweep(const SweepParams& P, int bits, int grid, int block, cudaStream_t s);
cudaError_t launch_serial(const SweepParams& P, int bits, cudaStream_t s);
cudaError_t launch_serial_batched(const SweepParams& P, int bits, cudaStream_t s);
void get_batched_kernels(int bits, bool serial, bool sym, bool lean, const void** prepare,
                         const void** sweep, const void** pairs);
cudaError_t launch_graph_pairs(const uint32_t* mate, const int64_t* vbase, uint64_t num_graphs,
                               uint64_t n, uint64_t* graph_pairs, int grid, cudaStream_t s);

// batch.cu: batched Skipper with a partition per member graph (local ids,
// warps-per-graph cap); every table is computed on the device
struct BatchParams {
  SweepParams P;           // the whole batch: n, nnz, offsets, nbrs, state, mate, work, err, spin_limit
  const int64_t* vbase;    // [G+1] first vertex of each graph
  const int64_t* ebase;    // [G+1] first entry of each graph
  uint64_t num_graphs;
  uint64_t* ubase;         // [G+1] first work unit of each graph (made on the device)
  uint64_t* sbase;         // [G+1] first state word of each graph (local ids, packed layouts)
  uint64_t* totals;        // [2]: units, state words
  uint32_t* gid;           // graph of each unit
  int64_t* part;           // per unit: first row (view coordinates), first entry (batch index)
  uint64_t grain;          // rows + entries per unit
  uint32_t wpg;            // most units per graph, 0 = no cap
  uint32_t local;          // 1: member graphs hold local ids
  uint64_t* graph_pairs;   // [G] matched pairs per graph, or null
};
struct BatchKernels {
  const void* plan;        // <<<1, batch_plan_threads()>>>(BatchParams)
  const void* prepare;     // (BatchParams, int states)
  const void* sweep;       // (BatchParams); the serial kernel takes one thread per graph
  const void* pairs;       // (BatchParams)
};
void get_batch_kernels(int bits, bool local, bool serial, bool sym, bool lean, BatchKernels* k);
int batch_sweep_blocks_per_sm(int bits, bool local, bool sym, bool lean, int block_threads);
int batch_plan_threads();
// one verdict for the whole batch in 9 counters (mm_verdict order after flags)
cudaError_t launch_validate_batch(const BatchParams& B, unsigned long long* counters, int grid,
                                  cudaStream_t s);

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
