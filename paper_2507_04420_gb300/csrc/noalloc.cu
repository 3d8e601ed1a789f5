// noalloc.cu -- mm_skipper_static: the matching pass without any device
// allocation.
//
// Some callers cannot allocate device memory while they work: a host program
// that hands all device memory to its own pool up front and forbids allocation
// afterwards, a latency-bound serving loop that must not pay for or risk a
// cudaMalloc per request, or a plug-in that runs inside someone else's process
// where the host owns the allocator.  This entry point gives them the pass with
// its scratch -- the packed byte states, the merge-path partition table and the
// work counter / error word -- in one fixed array that lives in this file and
// is reserved when the library is loaded.  The caller still passes the CSR and
// the mate array.
//
// The array holds kStaticBytes on every GPU that loads the library, until the
// process exits.  Host code never uses the array's name as an address: every
// call asks the runtime for the array's device address on the current device
// (cudaGetSymbolAddress) and hands that to the kernels.  Asking at every call,
// rather than once per device, keeps the address right for whatever context is
// current, also after cudaDeviceReset or in a context that is not the device's
// primary one (each context holds its own copy of the array); the first call in
// a context loads the library's device code there, so make it before any
// stream capture.  Every call reuses the same array: the preparation kernel
// clears the states, the work counter and the error word at the start of each
// call, and two calls whose work overlaps on the GPU (for example, from two
// host threads on two streams) race on it.
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "internal.h"
#include "skipper.h"

using namespace skp;

namespace {

constexpr uint64_t kStaticBytes = 8ull << 20;  // 8 MiB per device
constexpr uint64_t kCtrlBytes = 256;           // work counter, error word
constexpr uint64_t kMaxUnits = 32767;          // merge-path units per call
constexpr uint64_t kPartBytes = (kMaxUnits + 1) * 2 * sizeof(int64_t);
constexpr uint64_t kStateWords = (kStaticBytes - kCtrlBytes - kPartBytes) / sizeof(uint32_t);
static_assert(kStateWords * 4 == MM_STATIC_MAX_VERTICES, "capacity in skipper.h is out of date");

// The fixed scratch: [control | partition table | packed byte states].
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Device address of the scratch in the current context.
cudaError_t scratch_here(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" mm_status mm_skipper_static(uint64_t n, uint64_t nnz, const int64_t* d_offsets,
                                       const uint32_t* d_nbrs, uint32_t* d_mate,
                                       const mm_options* o, void* cuda_stream) {
  mm_options d;
  mm_default_options(&d);
  if (!o) o = &d;
  if (n > MM_STATIC_MAX_VERTICES) {
    set_error_message("mm_skipper_static: n = %llu exceeds the fixed scratch capacity of %llu vertices",
                      (unsigned long long)n, (unsigned long long)MM_STATIC_MAX_VERTICES);
    return MM_ERR_ARG;
  }
  auto reject = [](mm_status st, const char* why) {
    set_error_message("mm_skipper_static: %s", why);
    return st;
  };
  if (!d_offsets) return reject(MM_ERR_ARG, "null offsets");
  if (nnz && !d_nbrs) return reject(MM_ERR_ARG, "null nbrs with nnz > 0");
  if (n && !d_mate) return reject(MM_ERR_ARG, "null mate");
  if (nnz && (reinterpret_cast<uintptr_t>(d_nbrs) & 15u)) return reject(MM_ERR_ARG, "nbrs must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(d_offsets) & 7u) return reject(MM_ERR_ARG, "offsets must be 8-byte aligned");
  if (o->status_bits != 0 && o->status_bits != 8)
    return reject(MM_ERR_UNSUPPORTED, "only the byte state layout (status_bits 0 or 8) fits the fixed scratch");
  if (o->timing || o->use_graph || o->nosync || o->l2_persist)
    return reject(MM_ERR_UNSUPPORTED, "timing, use_graph, nosync and l2_persist need a handle (mm_create_csr)");
  if (o->stats || o->stage_windows || o->symmetric || o->id_loads == MM_ID_LOADS_SELECTIVE)
    return reject(MM_ERR_UNSUPPORTED, "stats, stage_windows, symmetric and selective id loads need a handle "
                                      "(mm_create_csr)");
  if (o->id_loads > MM_ID_LOADS_SELECTIVE) return reject(MM_ERR_ARG, "id_loads must be 0, 1 or 2");
  if (o->unit_order > MM_ORDER_DISPERSED) return reject(MM_ERR_ARG, "unit_order must be 0, 1 or 2");
  uint64_t grain = o->grain ? o->grain : 2048;
  if (grain % 128) return reject(MM_ERR_ARG, "grain must be a multiple of 128");
  const uint64_t items = n + nnz;
  if ((items + grain - 1) / grain > kMaxUnits) {  // a coarser split fits the table
    grain = (items + kMaxUnits - 1) / kMaxUnits;
    grain = (grain + 127) / 128 * 128;
  }
  if (grain > (1ull << 24)) {
    set_error_message("mm_skipper_static: %llu rows + entries need more than %llu work units",
                      (unsigned long long)items, (unsigned long long)kMaxUnits);
    return MM_ERR_ARG;
  }
  const int block = o->block_threads ? (int)o->block_threads : 512;
  if (block < 32 || block > 512 || block % 32)
    return reject(MM_ERR_ARG, "block_threads must be a multiple of 32 in [32, 512]");
  if (o->poison_vertex > n) return reject(MM_ERR_ARG, "poison_vertex out of range");

  auto cuda_fail = [](const char* what, cudaError_t e) {
    set_error_message("mm_skipper_static: %s: %s", what, cudaGetErrorString(e));
    return MM_ERR_CUDA;
  };
  cudaError_t e;
  int dev = -1;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail("cudaGetDevice", e);
  unsigned char* base = nullptr;
  if ((e = scratch_here(&base)) != cudaSuccess) return cuda_fail("cudaGetSymbolAddress", e);
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail("cudaDeviceGetAttribute", e);
  int l2 = 0;
  if ((e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev)) != cudaSuccess)
    return cuda_fail("cudaDeviceGetAttribute", e);
  // byte states: 64 warps per SM and dispersed units by default when the state
  // array takes at most half the L2, as in mm_skipper
  const bool fits = l2 > 0 && 2 * (4 * packed_words(n, 8)) <= (uint64_t)l2;

  SweepParams P{};
  P.n = n;
  P.nnz = nnz;
  P.offsets = d_offsets;
  P.nbrs = d_nbrs;
  P.mate = d_mate;
  P.work = reinterpret_cast<unsigned long long*>(base);
  P.err = reinterpret_cast<uint32_t*>(base + 8);
  P.part = reinterpret_cast<int64_t*>(base + kCtrlBytes);
  P.state = reinterpret_cast<uint32_t*>(base + kCtrlBytes + kPartBytes);
  P.grain = grain;
  P.units = (items + grain - 1) / grain;
  P.spin_limit = o->spin_limit ? o->spin_limit : (1ull << 20);
  P.poison = o->poison_vertex;
  P.disperse = (o->unit_order == MM_ORDER_DISPERSED || (o->unit_order == MM_ORDER_AUTO && fits)) ? 1u : 0u;

  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if ((e = launch_prepare(P, 8, sms * 8, s, nullptr, 0)) != cudaSuccess) return cuda_fail("prepare launch", e);
  if (o->serial) {
    e = launch_serial(P, 8, s);
  } else {
    P.lean = sweep_lean(8, block, (int)o->blocks_per_sm, fits) ? 1u : 0u;
    const int per_sm = o->blocks_per_sm ? (int)o->blocks_per_sm : sweep_blocks_per_sm(8, block, P.lean != 0);
    e = launch_sweep(P, 8, sms * per_sm, block, s);
  }
  if (e != cudaSuccess) return cuda_fail("sweep launch", e);
  uint32_t err = 0;  // the call's device status, read back into host stack memory
  if ((e = cudaMemcpyAsync(&err, P.err, sizeof err, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail("status read", e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail("cudaStreamSynchronize", e);
  if (err & kErrTimeout) return reject(MM_ERR_TIMEOUT, "a wait on a reserved vertex ran past spin_limit");
  if (err & kErrBadId) return reject(MM_ERR_BAD_GRAPH, "a neighbour id >= n was met");
  set_error_message("");
  return MM_OK;
}
