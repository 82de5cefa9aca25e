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

}  // namespace es
