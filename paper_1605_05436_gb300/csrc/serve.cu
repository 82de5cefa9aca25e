// serve.cu -- the serving engine: a native scheduler thread that admits
// exact-sum requests into device slots by a memory budget and runs
// continuous-batching steps (serve_kernel.cu) until every request is done.
//
//   submit()  -> pending queue (any host thread)
//   scheduler -> admit while a slot is free and the budget allows (FIFO);
//                host-memory requests are staged with an async copy on the
//                copy stream; build a step with one chunk of every active
//                request (shortest chunks first in tile order), upload it and
//                launch it; complete each request as soon as the device has
//                published its result (a sequence number in pinned host
//                memory); recycle steps whose completion event has fired
//   poll()    <- completion records (id, status, result bits, timestamps)
//
// Up to SERVE_STEPS_IN_FLIGHT steps are in flight, so the host prepares the
// next steps while one runs.  A request's partial sum stays in its device
// slot accumulator from its first chunk to its last.  A request's chunk is
// the larger of the engine's chunk and 1/max_steps of the request, so that
// a large request finishes in at most max_steps steps however many others
// share them.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/exactsum.h"
#include "digits.cuh"
#include "serve.h"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

int elem_bytes(int d) { return d == EXACTSUM_F64 ? 8 : (d == EXACTSUM_F32 ? 4 : 2); }

struct Req {
  uint64_t id = 0;
  const void* x = nullptr;   // caller's pointer
  const char* xd = nullptr;  // device pointer of the data
  int64_t n = 0;
  int in = 0, out = 0, mode = 0;
  bool host = false;
  int64_t bytes = 0;         // bytes held against the budget
  int64_t pos = 0;           // elements issued so far
  int slot = -1;
  bool fresh = true;         // staged copy not yet waited on by the compute stream
  int64_t chunk = 0;         // elements per step for this request
  void* staged = nullptr;
  cudaEvent_t ready = nullptr;
  int64_t submit_ns = 0, admit_ns = 0;
};

struct StepBuf {
  es::ServeBlock* h_block = nullptr;  // pinned
  es::ServeBlock* d_block = nullptr;
  es::ServeDone* h_done = nullptr;    // pinned, SERVE_MAX_ITEMS, written by the device
  es::ServeDone* d_done = nullptr;    // device alias of h_done
  cudaEvent_t done = nullptr;
  bool busy = false;
  int64_t seq = 0;
  std::vector<std::pair<int, Req*>> finals;  // (item, request) completing in this step
};

}  // namespace

constexpr int SERVE_STEPS_IN_FLIGHT = 2;

struct exactsum_server {
  int device = 0, num_sms = 0, max_slots = 0;
  int64_t budget = 0, chunk = 0, tile = 0, max_steps = 0;
  cudaStream_t compute = nullptr, copy = nullptr;
  int64_t* slot_acc = nullptr;
  StepBuf bufs[SERVE_STEPS_IN_FLIGHT];
  int64_t step_seq = 0;

  std::thread th;
  std::atomic<bool> stop{false};
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;                     // guarded by mu
  std::vector<exactsum_completion> done;        // guarded by mu
  std::atomic<int64_t> outstanding{0};          // submitted, not yet completed
  std::atomic<uint64_t> next_id{1};
  std::atomic<int> failed{0};
  std::string error = "no error";               // guarded by mu
  // scheduler-owned
  std::vector<Req*> slots;
  std::vector<std::pair<int64_t, Req*>> cand;   // chunks of the step being built
  int64_t mem_used = 0;
  int rr = 0;
  std::atomic<int64_t> steps_launched{0};
  std::atomic<int64_t> peak_active{0};
};

namespace {

void complete(exactsum_server* s, Req* r, int status, uint64_t bits) {
  exactsum_completion c;
  std::memset(&c, 0, sizeof c);
  c.id = r->id;
  c.status = status;
  c.out_dtype = r->out;
  c.result_bits = bits;
  c.n = r->n;
  c.submit_ns = r->submit_ns;
  c.admit_ns = r->admit_ns;
  c.done_ns = now_ns();
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->done.push_back(c);
  }
  s->outstanding.fetch_sub(1);
  s->cv.notify_all();
}

void release(exactsum_server* s, Req* r) {
  if (r->slot >= 0) s->slots[r->slot] = nullptr;
  s->mem_used -= r->bytes;
  if (r->staged) cudaFreeAsync(r->staged, s->compute);
  if (r->ready) cudaEventDestroy(r->ready);
  delete r;
}

void fail_all(exactsum_server* s, const char* what, cudaError_t e) {
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->error = std::string(what) + ": " + cudaGetErrorString(e);
  }
  s->failed.store(1);
  for (auto& b : s->bufs) b.finals.clear();
  for (auto& r : s->slots)
    if (r) {
      complete(s, r, EXACTSUM_ECUDA, 0);
      delete r;
      r = nullptr;
    }
  std::deque<Req*> rest;
  {
    std::lock_guard<std::mutex> g(s->mu);
    rest.swap(s->pending);
  }
  for (Req* r : rest) {
    complete(s, r, EXACTSUM_ECUDA, 0);
    delete r;
  }
}

// Complete the requests of in-flight steps whose results the device has
// published (the sequence number is written after the bits, behind a
// system-scope fence; the acquire fence orders the two reads here).
bool harvest(exactsum_server* s) {
  bool progress = false;
  for (auto& b : s->bufs) {
    if (!b.busy || b.finals.empty()) continue;
    for (size_t k = 0; k < b.finals.size();) {
      const int item = b.finals[k].first;
      const volatile es::ServeDone* d = b.h_done + item;
      if (d->seq != (unsigned long long)b.seq) {
        ++k;
        continue;
      }
      std::atomic_thread_fence(std::memory_order_acquire);
      Req* r = b.finals[k].second;
      complete(s, r, EXACTSUM_OK, d->bits);
      release(s, r);
      b.finals[k] = b.finals.back();
      b.finals.pop_back();
      progress = true;
    }
  }
  return progress;
}

// Recycle finished steps (after their last results have been harvested).
bool retire(exactsum_server* s) {
  bool progress = false;
  for (;;) {
    StepBuf* oldest = nullptr;
    for (auto& b : s->bufs)
      if (b.busy && (!oldest || b.seq < oldest->seq)) oldest = &b;
    if (!oldest) break;
    cudaError_t q = cudaEventQuery(oldest->done);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) {
      fail_all(s, "serving step", q);
      return true;
    }
    harvest(s);
    if (!oldest->finals.empty()) {
      // the step has finished but a final item published nothing
      fail_all(s, "serving step finished without publishing a result", cudaErrorUnknown);
      return true;
    }
    oldest->busy = false;
    progress = true;
  }
  return progress;
}

bool admit(exactsum_server* s) {
  bool progress = false;
  for (;;) {
    Req* r = nullptr;
    {
      std::lock_guard<std::mutex> g(s->mu);
      if (s->pending.empty()) break;
      r = s->pending.front();
      int free_slot = -1;
      for (int i = 0; i < s->max_slots; ++i)
        if (!s->slots[i]) {
          free_slot = i;
          break;
        }
      // FIFO: the head waits for a slot and for room in the budget; a request
      // larger than the whole budget runs alone
      const bool fits = s->mem_used + r->bytes <= s->budget || s->mem_used == 0;
      if (free_slot < 0 || !fits) break;
      s->pending.pop_front();
      r->slot = free_slot;
    }
    r->admit_ns = now_ns();
    r->chunk = s->chunk;
    if (s->max_steps > 0) {
      // at most max_steps steps: round the per-step share up to whole tiles
      const int64_t share = (r->n + s->max_steps - 1) / s->max_steps;
      const int64_t tiles = (share + s->tile - 1) / s->tile;
      r->chunk = std::max(s->chunk, tiles * s->tile);
    }
    s->slots[r->slot] = r;
    s->mem_used += r->bytes;
    if (r->host) {
      cudaError_t e = cudaMallocAsync(&r->staged, (size_t)r->n * elem_bytes(r->in), s->copy);
      if (e != cudaSuccess) {
        cudaGetLastError();
        s->slots[r->slot] = nullptr;
        s->mem_used -= r->bytes;
        r->staged = nullptr;
        complete(s, r, EXACTSUM_ENOMEM, 0);
        delete r;
        progress = true;
        continue;
      }
      cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
      cudaMemcpyAsync(r->staged, r->x, (size_t)r->n * elem_bytes(r->in), cudaMemcpyHostToDevice, s->copy);
      cudaEventRecord(r->ready, s->copy);
      r->xd = (const char*)r->staged;
    } else {
      r->xd = (const char*)r->x;
    }
    int64_t active = 0;
    for (Req* q : s->slots) active += q ? 1 : 0;
    if (active > s->peak_active.load()) s->peak_active.store(active);
    progress = true;
  }
  return progress;
}

// Elements per tile of a chunk: one warp streams one tile at a few GB/s, so
// a chunk is spread over all the step kernel's warps (tiles of len / warps,
// whole multiples of 1,024 elements), between 2,048 elements (below which the
// per-tile merge dominates) and the engine's tile.
int64_t chunk_tile(const exactsum_server* s, int64_t len) {
  const int64_t warps = (int64_t)s->num_sms * es::SERVE_WARPS_PER_CTA;
  int64_t t = (len + warps - 1) / warps;
  t = (t + 1023) / 1024 * 1024;
  return std::min(s->tile, std::max<int64_t>(t, 2048));
}

bool launch_step(exactsum_server* s) {
  StepBuf* b = nullptr;
  for (auto& c : s->bufs)
    if (!c.busy) {
      b = &c;
      break;
    }
  if (!b) return false;
  // one chunk of every active request; shortest first in tile order, so that
  // small requests are rounded (and published) early in the step
  auto& cand = s->cand;
  cand.clear();
  for (int k = 0; k < s->max_slots && (int)cand.size() < es::SERVE_MAX_ITEMS; ++k) {
    Req* r = s->slots[(s->rr + k) % s->max_slots];
    if (r && r->pos < r->n) cand.emplace_back(std::min(r->chunk, r->n - r->pos), r);
  }
  if (cand.empty()) return false;
  std::stable_sort(cand.begin(), cand.end(),
                   [](const std::pair<int64_t, Req*>& a, const std::pair<int64_t, Req*>& c) {
                     return a.first < c.first;
                   });
  const int64_t seq = s->step_seq + 1;
  int nitems = 0;
  int64_t tiles = 0;
  for (auto& cr : cand) {
    Req* r = cr.second;
    const int64_t len = cr.first;
    es::ServeItem& it = b->h_block->items[nitems];
    it.x = r->xd + r->pos * elem_bytes(r->in);
    it.len = len;
    it.tile = chunk_tile(s, len);
    it.tile_base = tiles;
    it.ntiles = (len + it.tile - 1) / it.tile;
    it.slot = r->slot;
    it.in = r->in;
    it.out = r->out;
    it.mode = r->mode;
    it.final = (r->pos + len == r->n) ? 1 : 0;
    it.pad = 0;
    b->h_block->remaining[nitems] = (unsigned)it.ntiles;
    tiles += it.ntiles;
    if (r->host && r->fresh) {
      cudaStreamWaitEvent(s->compute, r->ready, 0);
      r->fresh = false;
    }
    r->pos += len;
    if (it.final) b->finals.emplace_back(nitems, r);
    ++nitems;
  }
  s->rr = (s->rr + 1) % s->max_slots;
  b->h_block->queue = 0;
  // the block up to the last used item (the counters precede the items)
  const size_t bytes = offsetof(es::ServeBlock, items) + (size_t)nitems * sizeof(es::ServeItem);
  cudaError_t e = cudaMemcpyAsync(b->d_block, b->h_block, bytes, cudaMemcpyHostToDevice, s->compute);
  es::ServeStep st;
  st.items = b->d_block->items;
  st.nitems = nitems;
  st.remaining = b->d_block->remaining;
  st.queue = &b->d_block->queue;
  st.slot_acc = s->slot_acc;
  st.done = b->d_done;
  st.seq = (unsigned long long)seq;
  if (e == cudaSuccess) e = es::serve_launch(st, s->num_sms, s->compute);
  if (e == cudaSuccess) e = cudaEventRecord(b->done, s->compute);
  if (e != cudaSuccess) {
    fail_all(s, "serving launch", e);
    return true;
  }
  b->busy = true;
  b->seq = seq;
  s->step_seq = seq;
  s->steps_launched.fetch_add(1);
  return true;
}

void scheduler(exactsum_server* s) {
  cudaSetDevice(s->device);
  while (!s->failed.load()) {
    bool progress = harvest(s);
    progress |= retire(s);
    if (s->failed.load()) break;
    progress |= admit(s);
    progress |= launch_step(s);
    if (s->failed.load()) break;
    if (!progress) {
      bool busy = false;
      for (auto& b : s->bufs) busy |= b.busy;
      if (!busy) {
        bool any_active = false;
        for (Req* r : s->slots) any_active |= (r != nullptr);
        std::unique_lock<std::mutex> g(s->mu);
        if (s->stop.load() && s->pending.empty() && !any_active) break;
        if (s->pending.empty() && !any_active)
          s->cv.wait_for(g, std::chrono::milliseconds(2));
      } else {
        std::this_thread::yield();
      }
    }
  }
}

exactsum_status server_fail(exactsum_server* s, exactsum_status st, const std::string& msg) {
  if (s) {
    std::lock_guard<std::mutex> g(s->mu);
    s->error = msg;
  }
  return st;
}

void server_free(exactsum_server* s) {
  for (auto& b : s->bufs) {
    if (b.h_block) cudaFreeHost(b.h_block);
    if (b.h_done) cudaFreeHost(b.h_done);
    cudaFree(b.d_block);
    if (b.done) cudaEventDestroy(b.done);
  }
  cudaFree(s->slot_acc);
  if (s->compute) cudaStreamDestroy(s->compute);
  if (s->copy) cudaStreamDestroy(s->copy);
}

}  // namespace

extern "C" {

exactsum_status exactsum_server_create(exactsum_server_t* out, int device, int max_slots,
                                       int64_t mem_budget_bytes, int64_t chunk_elems, int64_t tile_elems,
                                       int max_steps_per_request) {
  if (!out) return EXACTSUM_EINVAL;
  *out = nullptr;
  if (max_slots < 1 || max_slots > es::SERVE_MAX_ITEMS || mem_budget_bytes <= 0 || chunk_elems < 1 ||
      tile_elems < 64 || tile_elems % 64 || chunk_elems % tile_elems || max_steps_per_request < 0)
    return EXACTSUM_EINVAL;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return EXACTSUM_ECUDA;
  if (prop.major != 10 || prop.minor != 3) return EXACTSUM_EUNSUPPORTED;
  if (cudaSetDevice(device) != cudaSuccess) return EXACTSUM_ECUDA;
  auto* s = new (std::nothrow) exactsum_server();
  if (!s) return EXACTSUM_ENOMEM;
  s->device = device;
  s->num_sms = prop.multiProcessorCount;
  s->max_slots = max_slots;
  s->budget = mem_budget_bytes;
  s->chunk = chunk_elems;
  s->tile = tile_elems;
  s->max_steps = max_steps_per_request;
  s->slots.assign(max_slots, nullptr);
  bool ok = es::serve_configure() == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaMalloc(&s->slot_acc, (size_t)max_slots * es::ACC_WORDS * sizeof(int64_t)) == cudaSuccess;
  ok = ok && cudaMemset(s->slot_acc, 0, (size_t)max_slots * es::ACC_WORDS * sizeof(int64_t)) == cudaSuccess;
  for (auto& b : s->bufs) {
    ok = ok && cudaMallocHost(&b.h_block, sizeof(es::ServeBlock)) == cudaSuccess;
    ok = ok && cudaHostAlloc(&b.h_done, es::SERVE_MAX_ITEMS * sizeof(es::ServeDone), cudaHostAllocMapped) ==
                   cudaSuccess;
    if (ok) std::memset(b.h_done, 0, es::SERVE_MAX_ITEMS * sizeof(es::ServeDone));
    ok = ok && cudaHostGetDevicePointer((void**)&b.d_done, b.h_done, 0) == cudaSuccess;
    ok = ok && cudaMalloc(&b.d_block, sizeof(es::ServeBlock)) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    server_free(s);
    delete s;
    return EXACTSUM_ENOMEM;
  }
  s->th = std::thread(scheduler, s);
  *out = s;
  return EXACTSUM_OK;
}

exactsum_status exactsum_server_submit(exactsum_server_t s, const void* x, int64_t n, exactsum_dtype in_dtype,
                                       exactsum_dtype out_dtype, exactsum_round mode, int x_on_host, uint64_t* id_out) {
  if (!s) return EXACTSUM_EINVAL;
  if (in_dtype < 0 || in_dtype > 2 || out_dtype < 0 || out_dtype > 2 || mode < 0 || mode > 3)
    return server_fail(s, EXACTSUM_EINVAL, "unknown dtype or mode");
  if (n < 0 || n >= ((int64_t)1 << 48) || (n > 0 && !x))
    return server_fail(s, EXACTSUM_EINVAL, "bad input pointer or size");
  if (((uintptr_t)x) % elem_bytes(in_dtype)) return server_fail(s, EXACTSUM_EINVAL, "input not aligned");
  if (s->failed.load()) return server_fail(s, EXACTSUM_ECUDA, "server failed earlier");
  Req* r = new (std::nothrow) Req();
  if (!r) return EXACTSUM_ENOMEM;
  r->id = s->next_id.fetch_add(1);
  r->x = x;
  r->n = n;
  r->in = in_dtype;
  r->out = out_dtype;
  r->mode = mode;
  r->host = x_on_host != 0;
  r->bytes = n * elem_bytes(in_dtype) + es::ACC_WORDS * 8;
  r->submit_ns = now_ns();
  if (id_out) *id_out = r->id;
  s->outstanding.fetch_add(1);
  if (n == 0) {  // the empty sum needs no device work
    r->admit_ns = r->submit_ns;
    complete(s, r, EXACTSUM_OK, 0);
    delete r;
    return EXACTSUM_OK;
  }
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->pending.push_back(r);
  }
  s->cv.notify_all();
  return EXACTSUM_OK;
}

exactsum_status exactsum_server_poll(exactsum_server_t s, exactsum_completion* out, int max_out, int* count) {
  if (!s || !count || (max_out > 0 && !out)) return EXACTSUM_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  const int k = std::min<int>(max_out, (int)s->done.size());
  for (int i = 0; i < k; ++i) out[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + k);
  *count = k;
  return EXACTSUM_OK;
}

exactsum_status exactsum_server_drain(exactsum_server_t s, int64_t timeout_ms) {
  if (!s) return EXACTSUM_EINVAL;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  std::unique_lock<std::mutex> g(s->mu);
  while (s->outstanding.load() > 0) {
    if (s->cv.wait_until(g, deadline) == std::cv_status::timeout && s->outstanding.load() > 0) {
      s->error = "drain timed out";
      return EXACTSUM_ETIMEOUT;
    }
  }
  return s->failed.load() ? EXACTSUM_ECUDA : EXACTSUM_OK;
}

exactsum_status exactsum_server_stats(exactsum_server_t s, int64_t* steps, int64_t* peak_active,
                                      int64_t* outstanding) {
  if (!s) return EXACTSUM_EINVAL;
  if (steps) *steps = s->steps_launched.load();
  if (peak_active) *peak_active = s->peak_active.load();
  if (outstanding) *outstanding = s->outstanding.load();
  return EXACTSUM_OK;
}

int64_t exactsum_server_clock_ns(void) { return now_ns(); }

const char* exactsum_server_last_error(exactsum_server_t s) {
  if (!s) return "null server";
  std::lock_guard<std::mutex> g(s->mu);
  static thread_local std::string copy;
  copy = s->error;
  return copy.c_str();
}

exactsum_status exactsum_server_destroy(exactsum_server_t s) {
  if (!s) return EXACTSUM_OK;
  s->stop.store(true);
  s->cv.notify_all();
  // requests still in the system are completed first (the scheduler only
  // exits when nothing is pending or active)
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->compute);
  cudaStreamSynchronize(s->copy);
  server_free(s);
  delete s;
  return EXACTSUM_OK;
}

}  // extern "C"
