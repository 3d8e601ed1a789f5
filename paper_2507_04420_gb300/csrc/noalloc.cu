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
// process exits.  Its device address is looked up once per device, with that
// device current, on the first call made on it (cudaGetSymbolAddress); host
// code never uses the array's name as an address.  Every call reuses the same
// array: the preparation kernel clears the states, the work counter and the
// error word at the start of each call, and two calls whose work overlaps on
// the GPU (for example, from two host threads on two streams) race on it.
#include <cstdint>
#include <cstring>
#include <mutex>
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

constexpr int kMaxDevices = 64;
std::mutex g_lock;
unsigned char* g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once.
cudaError_t scratch_on(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_lock);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_dev_ptr[dev];
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
  if (!d_offsets || (nnz && !d_nbrs) || (n && !d_mate)) return MM_ERR_ARG;
  if (nnz && (reinterpret_cast<uintptr_t>(d_nbrs) & 15u)) return MM_ERR_ARG;
  if (o->status_bits != 0 && o->status_bits != 8) return MM_ERR_UNSUPPORTED;
  if (o->timing || o->use_graph || o->nosync || o->l2_persist) return MM_ERR_UNSUPPORTED;
  uint64_t grain = o->grain ? o->grain : 2048;
  if (grain % 128) return MM_ERR_ARG;
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
  if (block < 32 || block > 512 || block % 32) return MM_ERR_ARG;
  if (o->poison_vertex > n) return MM_ERR_ARG;

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MM_ERR_CUDA;
  unsigned char* base = nullptr;
  if (scratch_on(dev, &base) != cudaSuccess) return MM_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MM_ERR_CUDA;

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

  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (launch_prepare(P, 8, sms * 8, s, nullptr, 0) != cudaSuccess) return MM_ERR_CUDA;
  cudaError_t e;
  if (o->serial) {
    e = launch_serial(P, 8, s);
  } else {
    const int per_sm = o->blocks_per_sm ? (int)o->blocks_per_sm : sweep_blocks_per_sm(8, block);
    e = launch_sweep(P, 8, sms * per_sm, block, s);
  }
  if (e != cudaSuccess) return MM_ERR_CUDA;
  uint32_t err = 0;  // the call's device status, read back into host stack memory
  if (cudaMemcpyAsync(&err, P.err, sizeof err, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MM_ERR_CUDA;
  if (err & kErrTimeout) return MM_ERR_TIMEOUT;
  if (err & kErrBadId) return MM_ERR_BAD_GRAPH;
  return MM_OK;
}
