// handle.h -- the library handle and workspace helpers (host side).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/exactsum.h"
#include "internal.h"

// A reducer configuration of the segmented kernel.
struct es_seg_config {
  int warps = 8;        // warps per CTA
  int kind = 0;         // reducer form: 0 register streaming, 1 TMA ring
  int64_t tile = 0;     // elements per tile
  float ms = -1.0f;     // measured time per call (autotuner), -1 if unmeasured
};

// Everything a captured segmented-sum graph depends on.
struct es_graph_key {
  const void* x;
  const int64_t* off;
  int64_t S;
  int in, out, mode;
  void* results;
  int warps;
  int kind;
  int64_t tile;
};

struct es_graph_entry {
  es_graph_key key;
  cudaGraphExec_t exec;
};

struct exactsum_ctx {
  int device = 0;
  int num_sms = 0;
  int max_ctas = 0;                 // CTAs of the single-array kernel (one per SM)
  std::string last_error = "no error";

  // single-array workspace: partial accumulators and the last-CTA ticket
  int64_t* partials = nullptr;      // partial_rows x ACC_WORDS
  int partial_rows = 0;
  unsigned int* ticket = nullptr;
  unsigned long long* dev_status = nullptr;  // STATUS_* bits set by kernels

  // host-buffer pipeline (exactsum_sum_host)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_consumed[2] = {nullptr, nullptr};
  void* stage[2] = {nullptr, nullptr};
  size_t stage_bytes = 0;
  int64_t* host_acc = nullptr;      // ACC_WORDS
  void* d_result_tmp = nullptr;     // 8 bytes
  void* h_result_pinned = nullptr;  // 8 bytes, page-locked

  // condition-number-sensitive sum (truncated.cu): per-pass state
  unsigned long long* trunc_state = nullptr;       // device, 8 words
  unsigned long long* trunc_state_host = nullptr;  // page-locked copy

  // segmented workspace (see segmented.cu)
  int64_t seg_capacity = 0;
  int64_t* seg_acc = nullptr;       // seg_capacity x ACC_WORDS, zero between calls
  int64_t* seg_tile_base = nullptr; // seg_capacity + 1
  unsigned int* seg_remaining = nullptr;  // seg_capacity
  unsigned long long* seg_counters = nullptr;  // work-queue head and misc counters
  int64_t* seg_block_tiles = nullptr;
  int64_t seg_block_capacity = 0;
  int32_t* seg_tile_seg = nullptr;  // tile -> segment map
  int64_t seg_map_capacity = 0;
  std::map<int, es_seg_config> seg_tuning;      // key: in_dtype * 64 + ceil(log2 S)
  std::vector<es_graph_entry> seg_graphs;       // most recently used first
  cudaStream_t capture_stream = nullptr;
};

exactsum_status es_cuda_fail(exactsum_t h, cudaError_t e, const char* what);
exactsum_status es_check_common(exactsum_t h, const void* x, int64_t n, int in, int out, int mode,
                                const void* dst);
es::SumArgs es_make_sum_args(const void* x, int64_t n, int in_dtype);
exactsum_status es_workspace_init(exactsum_t h);
void es_workspace_free(exactsum_t h);
exactsum_status es_segment_workspace_reserve(exactsum_t h, int64_t segments);
void es_segment_free_extra(exactsum_t h);
exactsum_status es_sum_host_pipelined(exactsum_t h, const void* h_x, int64_t n, int in, int out,
                                      int mode, void* h_result, cudaStream_t stream);
