// serve.h -- device-side structures of the serving engine's step kernel.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace es {

constexpr int SERVE_MAX_ITEMS = 256;  // requests per step (= max slots)

// One chunk of one request inside a step.
struct ServeItem {
  const void* x;      // first element of the chunk (device memory)
  int64_t len;        // elements in the chunk
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

struct ServeStep {
  const ServeItem* items;
  int nitems;
  int64_t tile;                 // elements per tile
  unsigned int* remaining;      // per item
  unsigned long long* queue;
  int64_t* slot_acc;            // max_slots x ACC_WORDS, zero between requests
  uint64_t* results;            // max_slots result bits
};

cudaError_t serve_configure();
cudaError_t serve_launch(const ServeStep& st, int grid, cudaStream_t stream);

}  // namespace es
