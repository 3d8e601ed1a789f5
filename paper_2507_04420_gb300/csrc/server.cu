// server.cu -- the continuous-batching serving loop, in native code.
//
// Clients submit graphs that live in host memory and collect each result by
// ticket; one worker thread (no Python, no interpreter lock) admits requests
// in arrival order while their device footprint fits the budget, and whenever
// a compute slot is free launches one multi-graph pass (mm_skipper_multi) over
// everything admitted since the last launch, followed on the same stream by
// the exact checker (mm_validate_multi_async).  Two slots alternate, so a new
// batch is admitted and launched while the previous one is on the GPU.
//
// A request reaches the GPU one of two ways.  Small ones whose host arrays
// the device can address (page-locked memory, or any host memory on a device
// that walks the host's page tables) are read in place through the host link;
// their mate arrays share one device arena per launch.  The others are copied
// to their own stream-ordered device buffers on a copy stream.  Mate arrays
// come back on a second copy stream into the caller's host buffers; device
// buffers are released stream-ordered once the checker has passed them.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>
#include <cuda_runtime.h>
#include <time.h>

#include "internal.h"
#include "skipper.h"

namespace {

int64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

struct Req {
  uint64_t ticket = 0;
  uint64_t n = 0, nnz = 0;
  const int64_t* h_off = nullptr;
  const uint32_t* h_nb = nullptr;
  uint32_t* h_mate = nullptr;
  bool in_place = false;
  const int64_t* off = nullptr;   // device addresses read by the kernels
  const uint32_t* nb = nullptr;
  uint32_t* mate = nullptr;       // device mate (own buffer, or a slice of the arena)
  bool own = false;               // off / nb / mate are this request's device buffers
  uint64_t bytes = 0;
  int64_t submit_ns = 0;
};

struct Tick {
  int slot = 0;
  std::vector<Req> reqs;          // with their device buffers, released once the tick is done
  uint32_t* arena = nullptr;      // mates of the in-place requests
  cudaEvent_t checked = nullptr, back = nullptr;
};

}  // namespace

struct mm_server {
  mm_server_config cfg{};
  int device = 0;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaStream_t slot_stream[2] = {nullptr, nullptr};
  // the server's own stream-ordered pool: it keeps freed memory mapped (up to
  // the budget) instead of returning it at every synchronisation, so a
  // request's buffers rarely need fresh device pages
  cudaMemPool_t pool = nullptr;
  mm_multi* slot_multi[2] = {nullptr, nullptr};
  int slots = 2, next_slot = 0;
  std::vector<cudaEvent_t> event_pool;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req> inbox;
  std::unordered_map<uint64_t, mm_server_result> done;
  uint64_t next_ticket = 1;
  bool closing = false;
  mm_status failure = MM_OK;
  char failure_msg[256] = "";
  std::thread worker;

  std::vector<void*> orphans;      // device buffers of a failed launch (worker only)
  std::atomic<uint64_t> used{0};   // device bytes held by admitted requests (worker writes)
  std::atomic<uint64_t> ticks{0}, graphs{0};  // launches and graphs launched
};

namespace {

thread_local char s_err[256] = "";

mm_status sfail(mm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(s_err, sizeof s_err, fmt, ap);
  va_end(ap);
  skp::set_error_message("%s", s_err);
  return st;
}

cudaEvent_t take_event(mm_server* s) {
  if (!s->event_pool.empty()) {
    cudaEvent_t e = s->event_pool.back();
    s->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  return e;
}

void finish(mm_server* s, Req& r, mm_status st, const mm_verdict* v) {
  mm_server_result res{};
  res.status = st;
  res.in_place = r.in_place ? 1u : 0u;
  if (v) res.verdict = *v;
  res.submit_ns = r.submit_ns;
  res.done_ns = now_ns();
  std::lock_guard<std::mutex> lk(s->mu);
  s->done[r.ticket] = res;
}

// Device buffers of work that never reached a completed launch: the copy
// buffers of staged requests and the arena of a launch that failed part way.
// A failed launch may have enqueued work on them, so every server stream is
// waited for first.  Errors are ignored: the server is already failing.
void release_orphans(mm_server* s, std::vector<Req>& staged) {
  for (Req& r : staged)
    if (r.own) {
      s->orphans.push_back(const_cast<int64_t*>(r.off));
      s->orphans.push_back(const_cast<uint32_t*>(r.nb));
      s->orphans.push_back(r.mate);
      r.own = false;
    }
  if (s->orphans.empty()) return;
  for (cudaStream_t st : {s->h2d, s->d2h, s->slot_stream[0], s->slot_stream[1]})
    if (st) cudaStreamSynchronize(st);
  for (void* p : s->orphans)
    if (p) cudaFree(p);
  s->orphans.clear();
  cudaGetLastError();
}

// Everything the worker holds fails with `st` (a worker failure).
void fail_all(mm_server* s, std::deque<Req>& pending, std::vector<Req>& staged,
              std::deque<Tick>& inflight, mm_status st) {
  for (Tick& t : inflight) {   // buffers of launched work: released once every stream is done
    for (Req& r : t.reqs)
      if (r.own) {
        s->orphans.push_back(const_cast<int64_t*>(r.off));
        s->orphans.push_back(const_cast<uint32_t*>(r.nb));
        s->orphans.push_back(r.mate);
        r.own = false;
      }
    if (t.arena) s->orphans.push_back(t.arena);
    t.arena = nullptr;
  }
  release_orphans(s, staged);
  for (Req& r : pending) finish(s, r, st, nullptr);
  for (Req& r : staged) finish(s, r, st, nullptr);
  for (Tick& t : inflight)
    for (Req& r : t.reqs) finish(s, r, st, nullptr);
  std::lock_guard<std::mutex> lk(s->mu);
  for (Req& r : s->inbox) {
    mm_server_result res{};
    res.status = st;
    res.submit_ns = r.submit_ns;
    res.done_ns = now_ns();
    s->done[r.ticket] = res;
  }
  s->inbox.clear();
  s->cv_done.notify_all();
}

#define W_TRY(expr)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      snprintf(s->failure_msg, sizeof s->failure_msg, "%s: %s", #expr, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA;                  \
    }                                                                                     \
  } while (0)

// copy path: the request's own device buffers, filled on the copy stream
mm_status admit_copy(mm_server* s, Req& r) {
  r.own = true;   // whatever of the three is allocated belongs to the request
  W_TRY(cudaMallocFromPoolAsync((void**)&r.off, 8 * (r.n + 1), s->pool, s->h2d));
  W_TRY(cudaMallocFromPoolAsync((void**)&r.nb, 4 * (r.nnz ? r.nnz : 1), s->pool, s->h2d));
  W_TRY(cudaMallocFromPoolAsync((void**)&r.mate, 4 * (r.n ? r.n : 1), s->pool, s->h2d));
  W_TRY(cudaMemcpyAsync(const_cast<int64_t*>(r.off), r.h_off, 8 * (r.n + 1), cudaMemcpyHostToDevice, s->h2d));
  if (r.nnz)
    W_TRY(cudaMemcpyAsync(const_cast<uint32_t*>(r.nb), r.h_nb, 4 * r.nnz, cudaMemcpyHostToDevice, s->h2d));
  return MM_OK;
}

mm_status launch_tick(mm_server* s, std::vector<Req>& staged, std::deque<Tick>& inflight,
                      uint32_t** arena_out) {
  Tick t;
  t.slot = s->next_slot;
  s->next_slot = (s->next_slot + 1) % s->slots;
  cudaStream_t st = s->slot_stream[t.slot];
  mm_multi* multi = s->slot_multi[t.slot];
  cudaEvent_t copied = take_event(s), swept = take_event(s);
  t.checked = take_event(s);
  t.back = take_event(s);
  if (!copied || !swept || !t.checked || !t.back) {
    snprintf(s->failure_msg, sizeof s->failure_msg, "event creation failed");
    return MM_ERR_CUDA;
  }
  W_TRY(cudaEventRecord(copied, s->h2d));
  W_TRY(cudaStreamWaitEvent(st, copied, 0));
  // one device arena for the mates of the in-place requests
  uint64_t arena_n = 0;
  for (const Req& r : staged)
    if (r.in_place) arena_n += r.n;
  uint32_t* arena = nullptr;
  if (arena_n) {
    W_TRY(cudaMallocFromPoolAsync((void**)&arena, 4 * arena_n, s->pool, st));
    *arena_out = arena;
    uint64_t at = 0;
    for (Req& r : staged)
      if (r.in_place) {
        r.mate = arena + at;
        at += r.n;
      }
  }
  std::vector<mm_graph_desc> descs(staged.size());
  for (size_t i = 0; i < staged.size(); ++i) {
    const Req& r = staged[i];
    descs[i] = mm_graph_desc{r.n, r.nnz, r.off, r.nnz ? r.nb : nullptr, r.n ? r.mate : nullptr};
  }
  mm_options o = s->cfg.opts;
  o.nosync = 1;
  // requests read in place cross the host link: selective id loads unless
  // the configuration fixes the choice
  bool any_in_place = false;
  for (const Req& r : staged) any_in_place = any_in_place || r.in_place;
  if (o.id_loads == MM_ID_LOADS_AUTO && any_in_place) o.id_loads = MM_ID_LOADS_SELECTIVE;
  mm_status ms = mm_skipper_multi(multi, descs.size(), descs.data(), &o, st);
  if (ms != MM_OK) {
    snprintf(s->failure_msg, sizeof s->failure_msg, "mm_skipper_multi: %s", mm_last_error());
    return ms;
  }
  W_TRY(cudaEventRecord(swept, st));
  if (s->cfg.validate) {
    ms = mm_validate_multi_async(multi, descs.size(), descs.data(), st);
    if (ms != MM_OK) {
      snprintf(s->failure_msg, sizeof s->failure_msg, "mm_validate_multi_async: %s", mm_last_error());
      return ms;
    }
  }
  W_TRY(cudaEventRecord(t.checked, st));
  // results back to the callers' buffers once the pass is done; the device
  // buffers stay with the tick until complete() has seen its checker and
  // these copies finish, and are then released on the copy stream, so the
  // copies of later requests can reuse them without waiting on another stream
  W_TRY(cudaStreamWaitEvent(s->d2h, swept, 0));
  for (const Req& r : staged)
    if (r.n && r.h_mate)
      W_TRY(cudaMemcpyAsync(r.h_mate, r.mate, 4 * r.n, cudaMemcpyDeviceToHost, s->d2h));
  W_TRY(cudaEventRecord(t.back, s->d2h));
  t.arena = arena;
  *arena_out = nullptr;
  s->event_pool.push_back(copied);   // recorded work keeps the event; reuse is stream-ordered
  s->event_pool.push_back(swept);
  s->ticks += 1;
  s->graphs += staged.size();
  t.reqs.swap(staged);
  inflight.push_back(std::move(t));
  return MM_OK;
}

mm_status launch(mm_server* s, std::vector<Req>& staged, std::deque<Tick>& inflight) {
  uint32_t* arena = nullptr;
  const mm_status st = launch_tick(s, staged, inflight, &arena);
  if (st != MM_OK && arena) s->orphans.push_back(arena);
  return st;
}

// the oldest tick, once its checker and its copies back are done
mm_status complete(mm_server* s, Tick& t, bool* ready) {
  *ready = false;
  cudaError_t a = cudaEventQuery(t.checked), b = cudaEventQuery(t.back);
  if (a == cudaErrorNotReady || b == cudaErrorNotReady) return MM_OK;
  W_TRY(a);
  W_TRY(b);
  *ready = true;
  mm_multi* multi = s->slot_multi[t.slot];
  const mm_status pass = mm_multi_sync(multi, s->slot_stream[t.slot]);  // timeouts, bad ids
  std::vector<mm_verdict> v;
  if (s->cfg.validate && pass == MM_OK) {
    v.resize(t.reqs.size());
    const mm_status vs = mm_multi_verdicts(multi, t.reqs.size(), v.data());
    if (vs != MM_OK) {
      snprintf(s->failure_msg, sizeof s->failure_msg, "mm_multi_verdicts: %s", mm_last_error());
      return vs;
    }
  }
  for (Req& r : t.reqs)
    if (r.own) {   // the tick's work on them is done: free on the copy stream
      W_TRY(cudaFreeAsync(const_cast<int64_t*>(r.off), s->h2d));
      r.off = nullptr;
      W_TRY(cudaFreeAsync(const_cast<uint32_t*>(r.nb), s->h2d));
      r.nb = nullptr;
      W_TRY(cudaFreeAsync(r.mate, s->h2d));
      r.mate = nullptr;
      r.own = false;
    }
  if (t.arena) W_TRY(cudaFreeAsync(t.arena, s->h2d));
  t.arena = nullptr;
  for (size_t i = 0; i < t.reqs.size(); ++i) {
    finish(s, t.reqs[i], pass, v.empty() ? nullptr : &v[i]);
    s->used -= t.reqs[i].bytes;
  }
  s->event_pool.push_back(t.checked);
  s->event_pool.push_back(t.back);
  s->cv_done.notify_all();
  return MM_OK;
}

void worker_main(mm_server* s) {
  std::deque<Req> pending;
  std::vector<Req> staged;
  std::deque<Tick> inflight;
  mm_status st = cudaSetDevice(s->device) == cudaSuccess ? MM_OK : MM_ERR_CUDA;
  if (st != MM_OK) snprintf(s->failure_msg, sizeof s->failure_msg, "cudaSetDevice failed in the worker");
  std::vector<uint64_t> sizes;
  while (st == MM_OK) {
    bool busy = false, closing = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      while (!s->inbox.empty()) {
        pending.push_back(std::move(s->inbox.front()));
        s->inbox.pop_front();
      }
      closing = s->closing;
    }
    while (st == MM_OK && !inflight.empty()) {
      bool ready = false;
      st = complete(s, inflight.front(), &ready);
      if (!ready || st != MM_OK) break;
      inflight.pop_front();
      busy = true;
    }
    if (st != MM_OK) break;
    // admission: arrival order, no overtaking, within the budget and the tick limits
    uint64_t staged_bytes = 0;
    for (const Req& r : staged) staged_bytes += r.bytes;
    const uint64_t tick_room = s->used + s->cfg.max_bytes_per_tick - staged_bytes;
    const uint64_t room = tick_room < s->cfg.memory_bytes ? tick_room : s->cfg.memory_bytes;
    sizes.clear();
    for (const Req& r : pending) sizes.push_back(r.bytes);
    uint64_t k = 0, add = 0;
    const uint64_t max_graphs = s->cfg.max_graphs_per_tick > staged.size()
                                    ? s->cfg.max_graphs_per_tick - staged.size() : 0;
    mm_server_plan_admission(sizes.data(), sizes.size(), s->used, room, max_graphs, &k, &add);
    if (k == 0 && staged.empty() && inflight.empty() && !pending.empty() &&
        pending.front().bytes > s->cfg.max_bytes_per_tick) {
      k = 1;  // one request larger than a tick runs alone
      add = pending.front().bytes;
    }
    for (uint64_t i = 0; i < k && st == MM_OK; ++i) {
      Req r = std::move(pending.front());
      pending.pop_front();
      if (!r.in_place) st = admit_copy(s, r);
      staged.push_back(std::move(r));
      busy = true;
    }
    s->used += add;
    if (st == MM_OK && !staged.empty() && (int)inflight.size() < s->slots) {
      st = launch(s, staged, inflight);
      busy = true;
    }
    if (st != MM_OK) break;
    if (closing && pending.empty() && staged.empty() && inflight.empty()) {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->inbox.empty()) return;
    }
    if (!busy) {
      std::unique_lock<std::mutex> lk(s->mu);
      // with work on the GPU poll its events soon; otherwise sleep until a submit
      s->cv_work.wait_for(lk, std::chrono::microseconds(inflight.empty() ? 2000 : 20),
                          [&] { return !s->inbox.empty() || s->closing; });
    }
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->failure = st;
  }
  fail_all(s, pending, staged, inflight, st);
}

}  // namespace

extern "C" {

mm_status mm_server_device_bytes(uint64_t n, uint64_t nnz, uint32_t in_place, uint64_t* out) {
  if (!out) return sfail(MM_ERR_ARG, "null out");
  auto r = [](uint64_t b) { return (b + 511) / 512 * 512; };
  const uint64_t scratch = (n / 4 + 8) + n + 24 * ((n + nnz) / 1024 + 2);
  const uint64_t csr = in_place ? 0 : r(8 * (n + 1)) + r(4 * (nnz ? nnz : 1));
  *out = csr + r(4 * (n ? n : 1)) + r(scratch);
  return MM_OK;
}

mm_status mm_server_plan_admission(const uint64_t* sizes, uint64_t count, uint64_t used,
                                   uint64_t budget, uint64_t max_graphs, uint64_t* k_out,
                                   uint64_t* bytes_out) {
  if ((count && !sizes) || !k_out || !bytes_out) return sfail(MM_ERR_ARG, "null argument");
  uint64_t k = 0, add = 0;
  for (; k < count && k < max_graphs; ++k) {
    if (used + add + sizes[k] > budget) break;
    add += sizes[k];
  }
  *k_out = k;
  *bytes_out = add;
  return MM_OK;
}

mm_status mm_server_default_config(mm_server_config* c) {
  if (!c) return sfail(MM_ERR_ARG, "null config");
  memset(c, 0, sizeof *c);
  c->reserve_bytes = 8ull << 30;
  c->max_graphs_per_tick = 4096;
  c->max_bytes_per_tick = 32ull << 30;
  c->in_place_max_nnz = 1ull << 20;
  c->validate = 1;
  c->slots = 2;
  return mm_default_options(&c->opts);
}

mm_status mm_server_create(const mm_server_config* cfg, mm_server** out) {
  if (!cfg || !out) return sfail(MM_ERR_ARG, "null argument");
  *out = nullptr;
  if (cfg->slots < 1 || cfg->slots > 2) return sfail(MM_ERR_ARG, "slots must be 1 or 2");
  if (cfg->max_graphs_per_tick == 0) return sfail(MM_ERR_ARG, "max_graphs_per_tick = 0");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return sfail(MM_ERR_CUDA, "no CUDA device");
  }
  mm_server* s = new (std::nothrow) mm_server();
  if (!s) return sfail(MM_ERR_OOM, "host allocation failed");
  s->cfg = *cfg;
  s->slots = (int)cfg->slots;
  auto bail = [&](mm_status st, const char* what) {
    for (int i = 0; i < 2; ++i) {
      if (s->slot_multi[i]) mm_multi_destroy(s->slot_multi[i]);
      if (s->slot_stream[i]) cudaStreamDestroy(s->slot_stream[i]);
    }
    if (s->h2d) cudaStreamDestroy(s->h2d);
    if (s->d2h) cudaStreamDestroy(s->d2h);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return sfail(st, "mm_server_create: %s", what);
  };
  if (cudaGetDevice(&s->device) != cudaSuccess) return bail(MM_ERR_CUDA, "cudaGetDevice");
  if (s->cfg.memory_bytes == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return bail(MM_ERR_CUDA, "cudaMemGetInfo");
    s->cfg.memory_bytes = free_b > cfg->reserve_bytes ? free_b - cfg->reserve_bytes : 0;
  }
  {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
      s->pool = nullptr;
      return bail(MM_ERR_CUDA, "cudaMemPoolCreate");
    }
    uint64_t keep = s->cfg.memory_bytes;
    if (cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
      return bail(MM_ERR_CUDA, "cudaMemPoolSetAttribute");
  }
  if (cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking) != cudaSuccess)
    return bail(MM_ERR_CUDA, "stream creation");
  for (int i = 0; i < s->slots; ++i) {
    if (cudaStreamCreateWithFlags(&s->slot_stream[i], cudaStreamNonBlocking) != cudaSuccess)
      return bail(MM_ERR_CUDA, "stream creation");
    if (mm_multi_create(&s->slot_multi[i]) != MM_OK) return bail(MM_ERR_OOM, "mm_multi_create");
  }
  try {
    s->worker = std::thread(worker_main, s);
  } catch (...) {
    return bail(MM_ERR_OOM, "worker thread");
  }
  *out = s;
  return MM_OK;
}

mm_status mm_server_submit(mm_server* s, uint64_t n, uint64_t nnz, const int64_t* h_offsets,
                           const uint32_t* h_nbrs, uint32_t* h_mate_out, uint64_t* ticket) {
  if (!s || !ticket || !h_offsets || (nnz && !h_nbrs) || (n && !h_mate_out))
    return sfail(MM_ERR_ARG, "null argument");
  if (n > MM_MAX_VERTICES) return sfail(MM_ERR_ARG, "n exceeds MM_MAX_VERTICES");
  Req r;
  r.n = n;
  r.nnz = nnz;
  r.h_off = h_offsets;
  r.h_nb = h_nbrs;
  r.h_mate = h_mate_out;
  r.submit_ns = now_ns();
  if (nnz <= s->cfg.in_place_max_nnz) {  // in place when the device can address both arrays
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    void* d_off = nullptr;
    void* d_nb = nullptr;
    bool ok = cudaHostGetDevicePointer(&d_off, const_cast<int64_t*>(h_offsets), 0) == cudaSuccess;
    if (ok && nnz) ok = cudaHostGetDevicePointer(&d_nb, const_cast<uint32_t*>(h_nbrs), 0) == cudaSuccess;
    if (ok && ((reinterpret_cast<uintptr_t>(d_off) & 7u) || (reinterpret_cast<uintptr_t>(d_nb) & 15u)))
      ok = false;   // the kernels' load widths
    cudaGetLastError();
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    if (ok) {
      r.in_place = true;
      r.off = static_cast<const int64_t*>(d_off);
      r.nb = static_cast<const uint32_t*>(d_nb);
    }
  }
  mm_server_device_bytes(n, nnz, r.in_place ? 1u : 0u, &r.bytes);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->failure != MM_OK) return sfail(s->failure, "server failed: %s", s->failure_msg);
  if (s->closing) return sfail(MM_ERR_ARG, "server is closing");
  r.ticket = s->next_ticket++;
  *ticket = r.ticket;
  if (r.bytes > s->cfg.memory_bytes) {  // can never fit: completes at once
    mm_server_result res{};
    res.status = MM_ERR_OOM;
    res.in_place = r.in_place ? 1u : 0u;
    res.submit_ns = res.done_ns = r.submit_ns;
    s->done[r.ticket] = res;
    s->cv_done.notify_all();
    return MM_OK;
  }
  s->inbox.push_back(std::move(r));
  s->cv_work.notify_one();
  return MM_OK;
}

mm_status mm_server_wait(mm_server* s, uint64_t ticket, double timeout_s, mm_server_result* out) {
  if (!s || !out) return sfail(MM_ERR_ARG, "null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto have = [&] { return s->done.count(ticket) != 0; };
  if (timeout_s > 0) {
    s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), have);
  }
  auto it = s->done.find(ticket);
  if (it == s->done.end()) return MM_PENDING;
  *out = it->second;
  s->done.erase(it);
  return MM_OK;
}

mm_status mm_server_stats(mm_server* s, uint64_t* launches, uint64_t* graphs, uint64_t* device_bytes_held) {
  if (!s) return sfail(MM_ERR_ARG, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (launches) *launches = s->ticks;
  if (graphs) *graphs = s->graphs;
  if (device_bytes_held) *device_bytes_held = s->used;
  return MM_OK;
}

mm_status mm_server_destroy(mm_server* s) {
  if (!s) return MM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->closing = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();   // drains every queued request
  const mm_status failure = s->failure;
  if (s->h2d) cudaStreamSynchronize(s->h2d);   // the last launches' buffers are freed on it
  cudaStreamSynchronize(s->d2h);
  for (int i = 0; i < 2; ++i) {
    if (s->slot_stream[i]) cudaStreamSynchronize(s->slot_stream[i]);
    if (s->slot_multi[i]) mm_multi_destroy(s->slot_multi[i]);
    if (s->slot_stream[i]) cudaStreamDestroy(s->slot_stream[i]);
  }
  if (s->h2d) cudaStreamDestroy(s->h2d);
  if (s->d2h) cudaStreamDestroy(s->d2h);
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  if (s->pool) cudaMemPoolDestroy(s->pool);   // its memory goes back to the device
  char msg[256];
  snprintf(msg, sizeof msg, "%s", s->failure_msg);
  delete s;
  if (failure != MM_OK) return sfail(failure, "server failed: %s", msg);
  return MM_OK;
}

}  // extern "C"
