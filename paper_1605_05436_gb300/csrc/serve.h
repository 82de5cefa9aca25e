// serve.h -- device-side structures of the serving engine's step kernel.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace es {

constexpr int SERVE_MAX_ITEMS = 256;  // requests per step (= max slots)
constexpr int SERVE_WARPS_PER_CTA = 8;  // warps of the step kernel per CTA (one CTA per SM)

// One chunk of one request inside a step.
struct ServeItem {
  const void* x;      // first element of the chunk (device memory)
  int64_t len;        // elements in the chunk
  int64_t tile;       // elements per tile of this chunk
  int64_t tile_base;  // first tile of this chunk within the step
  int64_t ntiles;     // tiles of this chunk
  int32_t slot;       // accumulator slot of the request
  int32_t in, out, mode;
  int32_t final;      // 1 if the chunk completes the request
  int32_t pad;
};

// Per-step block uploaded by the host (one copy): queue head, per-item tile
// counters, items.
struct ServeBlock {
  unsigned long long queue;
  unsigned int remaining[SERVE_MAX_ITEMS];
  ServeItem items[SERVE_MAX_ITEMS];
};

// Completion record of one item, written by the device into pinned host
// memory as soon as the item's request is rounded: the result bits, then,
// after a system-scope fence, the step's sequence number, which the host
// polls.  A request completes without waiting for the rest of its step.
struct ServeDone {
  uint64_t bits;
  unsigned long long seq;
};

struct ServeStep {
  const ServeItem* items;
  int nitems;
  unsigned int* remaining;      // per item
  unsigned long long* queue;
  int64_t* slot_acc;            // max_slots x ACC_WORDS, zero between requests
  ServeDone* done;              // per item, pinned host memory (device alias)
  unsigned long long seq;       // this step's sequence number (> 0)
};

cudaError_t serve_configure();
cudaError_t serve_launch(const ServeStep& st, int grid, cudaStream_t stream);

// ---------------------------------------------------------------------------
// Resident express kernel: a kernel that stays on the express lane's SMs and
// takes requests from a ring in pinned host memory, so that a small request
// costs no launch.  The host writes a request's descriptor, then advances
// the published request count; worker warps take requests in ring order and
// claim their tiles with an atomic add on the request's own tile counter (in
// device memory, tagged with the request index, so that a counter reused by
// a newer request at the same ring position is never taken for the old
// one), and add each tile into the request's slot accumulator; the warp that
// completes a request's last tile rounds it and publishes the result.
// ---------------------------------------------------------------------------
constexpr int XRING = 4096;  // descriptors in the ring (power of two)
constexpr int XWORKER_WARPS = SERVE_WARPS_PER_CTA - 1;  // per CTA; the last warp polls

struct __align__(16) XDesc {
  const void* x;       // request input (device memory)
  int64_t n;           // elements
  int64_t tile;        // elements per tile
  int64_t ntiles;
  int64_t q;           // request index (ring position q % XRING), to detect reuse
  int32_t slot, in, out, mode;
  int64_t pad[2];
};

// In pinned, device-mapped host memory.
struct XQueue {
  unsigned long long tail_req;    // descriptors published (monotonic; written last by the host)
  int32_t stop;                   // 1: the kernel exits when idle
  int32_t alive;                  // CTAs of the resident kernel still running
  unsigned long long pad[6];
  XDesc ring[XRING];
};

struct XArgs {
  XQueue* q;                      // device alias of the pinned queue
  unsigned long long* tiles;      // device, XRING: per ring position, (request index << 32) | tiles claimed
  unsigned int* done;             // device: per slot, tiles finished of its current request
  int64_t* slot_acc;              // device: per slot accumulator
  ServeDone* results;             // pinned: per slot, result bits then the request index + 1
  long long idle_ns;              // a CTA that saw no new request for this long exits
  long long first_req;            // every request before this one is complete
};

cudaError_t serve_resident_configure();
cudaError_t serve_resident_launch(const XArgs& a, int grid, cudaStream_t stream);

}  // namespace es
