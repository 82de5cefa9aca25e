// serve.cu -- the serving engine: a native scheduler thread that admits
// exact-sum requests into device slots by a memory budget and runs
// continuous-batching steps (serve_kernel.cu) until every request is done.
//
//   submit()  -> pending queue (any host thread)
//   scheduler -> admit while a slot is free and the budget allows (FIFO);
//                host-memory requests are staged with an async copy on the
//                copy stream; then, by size, one of two lanes:
//     express lane (requests of at most express_max_bytes): build a step with
//                one chunk of every active express request (shortest chunks
//                first in tile order), upload it and launch it on the express
//                stream; complete each request as soon as the device has
//                published its result (a sequence number in pinned host
//                memory); recycle steps whose completion event has fired;
//     bulk lane (larger requests): one launch of the single-array sum kernel
//                per request on the bulk stream, on all SMs but the
//                express_sms that the bulk lane leaves to the express lane,
//                its rounded result stored straight into pinned host memory;
//                the request completes when its event has fired
//   poll()    <- completion records (id, status, result bits, timestamps)
//
// The two lanes run at the same time on disjoint SMs, so a small request
// never waits behind a large one (the head-of-line blocking of one launch
// per request on one stream), and large requests run on the fast
// single-array kernel.  Up to SERVE_STEPS_IN_FLIGHT express steps are in
// flight, so the host prepares the next step while one runs.  An express
// request's partial sum stays in its device slot accumulator from its first
// chunk to its last; its chunk is the larger of the engine's chunk and
// 1/max_steps of the request.
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
#include "handle.h"
#include "internal.h"
#include "segmented.h"
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
  bool bulk = false;         // bulk lane (one single-array launch)
  cudaEvent_t bulk_done = nullptr;
  int64_t xq = -1;           // resident express lane: request index once published
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
// Lane defaults: requests above 4 MiB of input take the bulk lane, which
// leaves 8 SMs to the express lane (measured on the 20k req/s stream: 8 SMs
// gave the lowest p99, the same p50 as 16).
constexpr int64_t SERVE_EXPRESS_MAX_BYTES = (int64_t)4 << 20;
constexpr int SERVE_EXPRESS_SMS = 8;

struct exactsum_server {
  int device = 0, num_sms = 0, max_slots = 0;
  int64_t budget = 0, chunk = 0, tile = 0, max_steps = 0;
  cudaStream_t compute = nullptr, copy = nullptr, bulk = nullptr;
  int64_t* slot_acc = nullptr;
  // lanes (exactsum_server_set_lanes), fixed once the first request arrives
  int64_t express_max_bytes = SERVE_EXPRESS_MAX_BYTES;
  int express_sms = SERVE_EXPRESS_SMS;
  std::atomic<bool> started{false};
  // bulk lane: the single-array kernel's workspace (its launches are ordered
  // on the bulk stream, so one suffices) and per-slot results in pinned,
  // device-mapped host memory
  int64_t* bulk_partials = nullptr;
  unsigned int* bulk_ticket = nullptr;
  unsigned long long* bulk_status = nullptr;
  uint64_t* h_bulk_res = nullptr;  // max_slots
  uint64_t* d_bulk_res = nullptr;  // device alias
  std::deque<Req*> bulk_inflight;  // launch order
  // resident express lane (serve_resident_kernel): request ring and results
  // in pinned, device-mapped host memory
  int resident = 1;
  es::XQueue* hq = nullptr;
  es::XQueue* dq = nullptr;
  unsigned long long* x_tiles = nullptr;    // device, XRING tagged tile counters
  unsigned int* x_done = nullptr;           // device, max_slots
  es::ServeDone* h_xres = nullptr;          // max_slots
  es::ServeDone* d_xres = nullptr;
  int64_t x_next_req = 0;
  std::deque<Req*> x_waiting;               // admitted, not yet published
  int64_t x_launches = 0;
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
  std::atomic<uint64_t> submitted{0};  // requests queued (monotonic)
};

// An idle scheduler keeps polling for new requests this long before it
// sleeps on the condition variable: a request that arrives in that window
// is admitted at once instead of after a thread wake-up (tens of
// microseconds).  The price is one host core busy while requests keep
// coming.
constexpr int64_t SERVE_IDLE_SPIN_NS = 2000000;

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
  // staging memory is freed on a stream that is past its last reader (the
  // resident kernel never ends while requests keep coming, so not on its
  // stream: its result being published means the input has been read)
  if (r->staged) cudaFreeAsync(r->staged, r->bulk ? s->bulk : (r->xq >= 0 ? s->copy : s->compute));
  if (r->ready) cudaEventDestroy(r->ready);
  if (r->bulk_done) cudaEventDestroy(r->bulk_done);
  delete r;
}

void fail_all(exactsum_server* s, const char* what, cudaError_t e) {
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->error = std::string(what) + ": " + cudaGetErrorString(e);
  }
  s->failed.store(1);
  for (auto& b : s->bufs) b.finals.clear();
  s->bulk_inflight.clear();
  s->x_waiting.clear();
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

// Complete bulk requests whose launch has finished (in launch order).
bool harvest_bulk(exactsum_server* s) {
  bool progress = false;
  while (!s->bulk_inflight.empty()) {
    Req* r = s->bulk_inflight.front();
    const cudaError_t q = cudaEventQuery(r->bulk_done);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) {
      fail_all(s, "serving bulk launch", q);
      return true;
    }
    s->bulk_inflight.pop_front();
    const volatile uint64_t* res = s->h_bulk_res + r->slot;
    const int w = elem_bytes(r->out);
    const uint64_t mask = w == 8 ? ~0ull : ((1ull << (8 * w)) - 1);
    complete(s, r, EXACTSUM_OK, *res & mask);
    release(s, r);
    progress = true;
  }
  return progress;
}

// One launch of the single-array sum for a bulk request: all SMs but the
// express lane's, the result rounded straight into the slot's word of pinned
// host memory.
bool launch_bulk(exactsum_server* s, Req* r) {
  es::SumArgs a = es_make_sum_args(r->xd, r->n, r->in);
  a.out = r->out;
  a.mode = r->mode;
  a.result = s->d_bulk_res + r->slot;
  a.acc = nullptr;
  a.partials = s->bulk_partials;
  a.ticket = s->bulk_ticket;
  a.status = s->bulk_status;
  cudaError_t e = cudaEventCreateWithFlags(&r->bulk_done, cudaEventDisableTiming);
  if (e == cudaSuccess && r->host) e = cudaStreamWaitEvent(s->bulk, r->ready, 0);
  const int ctas = std::max(1, s->num_sms - s->express_sms);
  if (e == cudaSuccess) e = es::launch_sum(r->in, a, ctas, s->bulk, nullptr);
  if (e == cudaSuccess) e = cudaEventRecord(r->bulk_done, s->bulk);
  if (e != cudaSuccess) {
    s->bulk_inflight.push_back(r);  // completed with an error by fail_all
    fail_all(s, "serving bulk launch", e);
    return false;
  }
  r->pos = r->n;
  s->bulk_inflight.push_back(r);
  return true;
}

// ---- resident express lane ----
constexpr long long SERVE_RESIDENT_IDLE_NS = 5000000;  // a resident CTA idle this long exits

// Elements per tile of a resident request: spread over the lane's worker
// warps, whole multiples of 1,024 elements, between 2,048 and the engine's tile.
int64_t resident_tile(const exactsum_server* s, int64_t len) {
  const int64_t warps = (int64_t)s->express_sms * es::XWORKER_WARPS;
  int64_t t = (len + warps - 1) / warps;
  t = (t + 1023) / 1024 * 1024;
  return std::min(s->tile, std::max<int64_t>(t, 2048));
}

// Launch the resident kernel if no CTA of it is alive.  The host has just
// published work (tail stores) and now reads the alive count; a CTA leaving
// first lowers the count and then reads the tail (both with system-scope
// fences), so at least one of the two sees the other's write.
bool ensure_resident(exactsum_server* s) {
  std::atomic_thread_fence(std::memory_order_seq_cst);
  if (__atomic_load_n(&s->hq->alive, __ATOMIC_SEQ_CST) > 0) return true;
  const int grid = std::max(1, std::min(s->num_sms, s->express_sms));
  __atomic_fetch_add(&s->hq->alive, grid, __ATOMIC_SEQ_CST);
  es::XArgs a;
  a.q = s->dq;
  a.tiles = s->x_tiles;
  a.done = s->x_done;
  a.slot_acc = s->slot_acc;
  a.results = s->d_xres;
  a.idle_ns = SERVE_RESIDENT_IDLE_NS;
  // the oldest request not yet complete: the kernel's warps scan from there
  a.first_req = s->x_next_req;
  for (Req* o : s->slots)
    if (o && o->xq >= 0) a.first_req = std::min<long long>(a.first_req, o->xq);
  const cudaError_t e = es::serve_resident_launch(a, grid, s->compute);
  if (e != cudaSuccess) {
    fail_all(s, "resident kernel launch", e);
    return false;
  }
  ++s->x_launches;
  s->steps_launched.fetch_add(1);
  return true;
}

// Publish admitted express requests whose input is ready, in order: write
// the descriptor, then advance the request and tile counts (release).
bool publish_resident(exactsum_server* s) {
  bool progress = false;
  while (!s->x_waiting.empty()) {
    Req* r = s->x_waiting.front();
    if (r->host) {
      const cudaError_t q = cudaEventQuery(r->ready);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        fail_all(s, "serving staging copy", q);
        return true;
      }
    }
    // the ring entry must not belong to a request still in flight
    int64_t oldest = s->x_next_req;
    for (Req* o : s->slots)
      if (o && o->xq >= 0) oldest = std::min(oldest, o->xq);
    if (s->x_next_req - oldest >= es::XRING) break;
    s->x_waiting.pop_front();
    const int64_t tile = resident_tile(s, r->n);
    const int64_t ntiles = (r->n + tile - 1) / tile;
    es::XDesc& d = s->hq->ring[s->x_next_req & (es::XRING - 1)];
    d.x = r->xd;
    d.n = r->n;
    d.tile = tile;
    d.ntiles = ntiles;
    d.q = s->x_next_req;
    d.slot = r->slot;
    d.in = r->in;
    d.out = r->out;
    d.mode = r->mode;
    r->xq = s->x_next_req;
    r->pos = r->n;
    ++s->x_next_req;
    __atomic_store_n(&s->hq->tail_req, (unsigned long long)s->x_next_req, __ATOMIC_RELEASE);
    progress = true;
  }
  if (progress && !ensure_resident(s)) return true;
  return progress;
}

// Complete resident requests whose result the device has published.
bool harvest_resident(exactsum_server* s) {
  bool progress = false;
  for (int k = 0; k < s->max_slots; ++k) {
    Req* r = s->slots[k];
    if (!r || r->xq < 0) continue;
    const volatile es::ServeDone* d = s->h_xres + k;
    if (d->seq != (unsigned long long)(r->xq + 1)) continue;
    std::atomic_thread_fence(std::memory_order_acquire);
    complete(s, r, EXACTSUM_OK, d->bits);
    release(s, r);
    progress = true;
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
    r->bulk = s->express_max_bytes >= 0 && r->n * elem_bytes(r->in) > s->express_max_bytes;
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
    if (r->bulk) {
      if (!launch_bulk(s, r)) return true;
    } else if (s->resident) {
      s->x_waiting.push_back(r);
    }
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
  if (s->resident) return false;
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
    if (r && !r->bulk && r->pos < r->n) cand.emplace_back(std::min(r->chunk, r->n - r->pos), r);
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
  // while the bulk lane holds its SMs, the step runs on the express lane's
  const int grid = s->bulk_inflight.empty() ? s->num_sms : std::max(1, std::min(s->num_sms, s->express_sms));
  if (e == cudaSuccess) e = es::serve_launch(st, grid, s->compute);
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
  int64_t idle_since = -1;
  while (!s->failed.load()) {
    bool progress = harvest(s);
    progress |= harvest_bulk(s);
    progress |= harvest_resident(s);
    progress |= retire(s);
    if (s->failed.load()) break;
    progress |= admit(s);
    progress |= publish_resident(s);
    progress |= launch_step(s);
    if (s->failed.load()) break;
    if (progress) idle_since = -1;
    if (!progress) {
      bool busy = !s->bulk_inflight.empty() || !s->x_waiting.empty();
      for (auto& b : s->bufs) busy |= b.busy;
      for (Req* r : s->slots) busy |= (r && r->xq >= 0);
      if (!busy) {
        bool any_active = false;
        for (Req* r : s->slots) any_active |= (r != nullptr);
        if (!any_active && !s->stop.load()) {
          // spin a while for the next request before sleeping
          const int64_t now = now_ns();
          if (idle_since < 0) idle_since = now;
          if (now - idle_since < SERVE_IDLE_SPIN_NS) {
            const uint64_t seen = s->submitted.load(std::memory_order_acquire);
            while (s->submitted.load(std::memory_order_acquire) == seen && !s->stop.load() &&
                   now_ns() - idle_since < SERVE_IDLE_SPIN_NS) {
            }
            continue;
          }
        }
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
  cudaFree(s->bulk_partials);
  cudaFree(s->bulk_ticket);
  cudaFree(s->bulk_status);
  if (s->h_bulk_res) cudaFreeHost(s->h_bulk_res);
  if (s->hq) cudaFreeHost(s->hq);
  if (s->h_xres) cudaFreeHost(s->h_xres);
  cudaFree(s->x_tiles);
  cudaFree(s->x_done);
  if (s->compute) cudaStreamDestroy(s->compute);
  if (s->copy) cudaStreamDestroy(s->copy);
  if (s->bulk) cudaStreamDestroy(s->bulk);
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
  ok = ok && cudaStreamCreateWithFlags(&s->bulk, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaMalloc(&s->bulk_partials, (size_t)s->num_sms * es::ACC_WORDS * sizeof(int64_t)) == cudaSuccess;
  ok = ok && cudaMalloc(&s->bulk_ticket, sizeof(unsigned int)) == cudaSuccess;
  ok = ok && cudaMemset(s->bulk_ticket, 0, sizeof(unsigned int)) == cudaSuccess;
  ok = ok && cudaMalloc(&s->bulk_status, sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMemset(s->bulk_status, 0, sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaHostAlloc(&s->h_bulk_res, (size_t)max_slots * sizeof(uint64_t), cudaHostAllocMapped) == cudaSuccess;
  ok = ok && cudaHostGetDevicePointer((void**)&s->d_bulk_res, s->h_bulk_res, 0) == cudaSuccess;
  ok = ok && es::serve_resident_configure() == cudaSuccess;
  // the library's kernels are loaded now, not at a first launch next to a
  // running resident kernel (a launch that has to load its module waits
  // for the kernels already running, and the resident kernel leaves only
  // when requests pause)
  ok = ok && es::preload_sum_kernels() == cudaSuccess;
  ok = ok && es::seg_preload() == cudaSuccess;
  ok = ok && es::trunc_preload() == cudaSuccess;
  ok = ok && cudaHostAlloc(&s->hq, sizeof(es::XQueue), cudaHostAllocMapped) == cudaSuccess;
  if (ok) std::memset(s->hq, 0, sizeof(es::XQueue));
  ok = ok && cudaHostGetDevicePointer((void**)&s->dq, s->hq, 0) == cudaSuccess;
  ok = ok && cudaHostAlloc(&s->h_xres, (size_t)max_slots * sizeof(es::ServeDone), cudaHostAllocMapped) == cudaSuccess;
  if (ok) std::memset(s->h_xres, 0, (size_t)max_slots * sizeof(es::ServeDone));
  ok = ok && cudaHostGetDevicePointer((void**)&s->d_xres, s->h_xres, 0) == cudaSuccess;
  ok = ok && cudaMalloc(&s->x_tiles, es::XRING * sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMemset(s->x_tiles, 0, es::XRING * sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMalloc(&s->x_done, (size_t)max_slots * sizeof(unsigned int)) == cudaSuccess;
  ok = ok && cudaMemset(s->x_done, 0, (size_t)max_slots * sizeof(unsigned int)) == cudaSuccess;
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
  s->started.store(true);
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
  s->submitted.fetch_add(1, std::memory_order_release);
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

exactsum_status exactsum_server_set_lanes(exactsum_server_t s, int64_t express_max_bytes, int express_sms,
                                         int resident) {
  if (!s) return EXACTSUM_EINVAL;
  if (s->started.load()) return server_fail(s, EXACTSUM_EINVAL, "lanes must be set before the first submission");
  if (express_sms < 1 || express_sms >= s->num_sms)
    return server_fail(s, EXACTSUM_EINVAL, "express_sms must be in [1, SMs)");
  if (resident != 0 && resident != 1) return server_fail(s, EXACTSUM_EINVAL, "resident must be 0 or 1");
  s->express_max_bytes = express_max_bytes;
  s->express_sms = express_sms;
  s->resident = resident;
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
  // the resident kernel leaves at its next look at the queue
  if (s->hq) __atomic_store_n(&s->hq->stop, 1, __ATOMIC_SEQ_CST);
  cudaStreamSynchronize(s->compute);
  cudaStreamSynchronize(s->copy);
  cudaStreamSynchronize(s->bulk);
  server_free(s);
  delete s;
  return EXACTSUM_OK;
}

}  // extern "C"
