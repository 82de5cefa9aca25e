// segmented.h -- arguments and launch entry of the segmented-sum kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace es {

enum : int { CNT_QUEUE = 0, CNT_TOTAL = 1 };

struct SegArgs {
  const void* x;                 // elements (element-aligned)
  const int64_t* off;            // S + 1 CSR offsets (device)
  int64_t S;
  int out, mode;
  void* results;                 // S elements of the output format
  int64_t tile;                  // elements per tile
  int64_t* block_tiles;          // ceil(S / 1024) per-block tile sums, then their scan
  int64_t* tile_base;            // S + 1: first tile of each segment
  int32_t* tile_seg;             // map_capacity: segment of each tile
  int64_t map_capacity;
  unsigned int* remaining;       // S: tiles not yet retired
  int64_t* seg_acc;              // S x ACC_WORDS, zero between calls
  unsigned long long* counters;  // CNT_* words
  unsigned long long* status;    // device status word (STATUS_* bits)
};

// Reducer forms: register streaming (warps choice 0 or 1) or the TMA ring.
enum : int { SEG_KIND_REGISTER = 0, SEG_KIND_TMA = 1, SEG_KIND_WINDOW = 2 };

// Enqueue the four kernels of one segmented sum on `st`.
cudaError_t seg_enqueue(int in_dt, const SegArgs& a, int warps, int kind, int num_sms, cudaStream_t st);
// Warps per CTA of the reducer for a dtype: register form choice 0 or 1;
// choice 2 is the TMA form's fixed shape, choice 3 the windowed form's.
int seg_warps_choice(int in_dt, int idx);
// Load and configure every segmented kernel on the current device now.
cudaError_t seg_preload();

}  // namespace es
