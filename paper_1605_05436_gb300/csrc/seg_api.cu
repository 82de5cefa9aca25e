// seg_api.cu -- C ABI of the segmented sum: workspace, CUDA-graph cache,
// autotuner and its JSON cache, device status word, per-segment baseline.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/exactsum.h"
#include "digits.cuh"
#include "handle.h"
#include "internal.h"
#include "segmented.h"

namespace {

int elem_bytes(int d) { return d == EXACTSUM_F64 ? 8 : (d == EXACTSUM_F32 ? 4 : 2); }

int ceil_log2(int64_t v) {
  int k = 0;
  while (((int64_t)1 << k) < v) ++k;
  return k;
}

exactsum_status fail(exactsum_t h, exactsum_status st, const std::string& msg) {
  if (h) h->last_error = msg;
  return st;
}

// Default reducer configuration: 256 KiB tiles, the smaller CTA.
es_seg_config default_config(int in) {
  es_seg_config c;
  c.warps = es::seg_warps_choice(in, 0);
  c.tile = (int64_t)(256 << 10) / elem_bytes(in);
  c.ms = -1.0f;
  return c;
}

es_seg_config lookup_config(exactsum_t h, int in, int64_t S) {
  const int key = in * 64 + ceil_log2(S);
  auto it = h->seg_tuning.find(key);
  if (it != h->seg_tuning.end()) return it->second;
  return default_config(in);
}

void clear_graphs(exactsum_t h) {
  for (auto& g : h->seg_graphs) cudaGraphExecDestroy(g.exec);
  h->seg_graphs.clear();
}

// Workspace for S segments and the tile map of one configuration.
exactsum_status ensure_workspace(exactsum_t h, int64_t S, int in, int64_t tile, bool capturing) {
  const int64_t nblocks = (S + 1023) / 1024;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  // a tile map that covers any input that fits in device memory
  const int64_t map_need = S + (int64_t)(total_b / (size_t)elem_bytes(in) / (size_t)tile) + 1;
  const bool grow = S > h->seg_capacity || nblocks > h->seg_block_capacity || map_need > h->seg_map_capacity;
  if (!grow) return EXACTSUM_OK;
  if (capturing)
    return fail(h, EXACTSUM_EINVAL,
                "segmented workspace must grow, which cannot happen during stream capture: "
                "call once outside capture first (or pass max_segments_hint)");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return es_cuda_fail(h, e, "cudaDeviceSynchronize");
  clear_graphs(h);
  exactsum_status st = es_segment_workspace_reserve(h, std::max(S, h->seg_capacity));
  if (st != EXACTSUM_OK) return st;
  if (nblocks > h->seg_block_capacity) {
    cudaFree(h->seg_block_tiles);
    h->seg_block_tiles = nullptr;
    h->seg_block_capacity = 0;
    if ((e = cudaMalloc(&h->seg_block_tiles, (size_t)nblocks * sizeof(int64_t))) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaMalloc(block tiles)");
    h->seg_block_capacity = nblocks;
  }
  if (map_need > h->seg_map_capacity) {
    cudaFree(h->seg_tile_seg);
    h->seg_tile_seg = nullptr;
    h->seg_map_capacity = 0;
    if ((e = cudaMalloc(&h->seg_tile_seg, (size_t)map_need * sizeof(int32_t))) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaMalloc(tile map)");
    h->seg_map_capacity = map_need;
  }
  return EXACTSUM_OK;
}

es::SegArgs make_args(exactsum_t h, const void* x, const int64_t* off, int64_t S, int out, int mode,
                      void* results, int64_t tile) {
  es::SegArgs a{};
  a.x = x;
  a.off = off;
  a.S = S;
  a.out = out;
  a.mode = mode;
  a.results = results;
  a.tile = tile;
  a.block_tiles = h->seg_block_tiles;
  a.tile_base = h->seg_tile_base;
  a.tile_seg = h->seg_tile_seg;
  a.map_capacity = h->seg_map_capacity;
  a.remaining = h->seg_remaining;
  a.seg_acc = h->seg_acc;
  a.counters = h->seg_counters;
  a.status = h->dev_status;
  return a;
}

exactsum_status check_seg_args(exactsum_t h, const void* x, const int64_t* off, int64_t S, int in, int out,
                               int mode, const void* results) {
  exactsum_status st = es_check_common(h, x, 0, in, out, mode, results);
  if (st != EXACTSUM_OK) return st;
  if (S < 0 || S >= ((int64_t)1 << 31)) return fail(h, EXACTSUM_EINVAL, "num_segments out of range [0, 2^31)");
  if (S > 0 && !off) return fail(h, EXACTSUM_EINVAL, "null offsets");
  if (((uintptr_t)off) % 8) return fail(h, EXACTSUM_EINVAL, "offsets not 8-byte aligned");
  if (((uintptr_t)x) % elem_bytes(in)) return fail(h, EXACTSUM_EINVAL, "input not aligned to its element size");
  if (((uintptr_t)results) % elem_bytes(out)) return fail(h, EXACTSUM_EINVAL, "results not aligned");
  return EXACTSUM_OK;
}

exactsum_status run_segmented(exactsum_t h, const void* x, const int64_t* off, int64_t S, int in, int out,
                              int mode, void* results, cudaStream_t stream, const es_seg_config& cfg,
                              bool use_graph) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &cs);
  if (e != cudaSuccess) return es_cuda_fail(h, e, "cudaStreamIsCapturing");
  const bool capturing = cs != cudaStreamCaptureStatusNone;
  exactsum_status st = ensure_workspace(h, S, in, cfg.tile, capturing);
  if (st != EXACTSUM_OK) return st;
  es::SegArgs a = make_args(h, x, off, S, out, mode, results, cfg.tile);
  if (capturing || !use_graph) {
    e = es::seg_enqueue(in, a, cfg.warps, cfg.kind, h->num_sms, stream);
    if (e != cudaSuccess) return es_cuda_fail(h, e, "segmented launch");
    return EXACTSUM_OK;
  }
  es_graph_key key{};  // value-initialised: padding bytes compare equal
  key.x = x;
  key.off = off;
  key.S = S;
  key.in = in;
  key.out = out;
  key.mode = mode;
  key.results = results;
  key.warps = cfg.warps;
  key.kind = cfg.kind;
  key.tile = cfg.tile;
  cudaGraphExec_t exec = nullptr;
  for (size_t i = 0; i < h->seg_graphs.size(); ++i) {
    if (std::memcmp(&h->seg_graphs[i].key, &key, sizeof key) == 0) {
      exec = h->seg_graphs[i].exec;
      if (i != 0) std::swap(h->seg_graphs[i], h->seg_graphs[0]);  // most recent first
      break;
    }
  }
  if (!exec) {
    if (!h->capture_stream) {
      if ((e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return es_cuda_fail(h, e, "cudaStreamCreate(capture)");
    }
    if ((e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaStreamBeginCapture");
    cudaError_t le = es::seg_enqueue(in, a, cfg.warps, cfg.kind, h->num_sms, h->capture_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->capture_stream, &graph);
    if (le != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return es_cuda_fail(h, le, "segmented launch (capture)");
    }
    if (e != cudaSuccess) return es_cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return es_cuda_fail(h, e, "cudaGraphInstantiate");
    if (h->seg_graphs.size() >= 16) {
      cudaGraphExecDestroy(h->seg_graphs.back().exec);
      h->seg_graphs.pop_back();
    }
    h->seg_graphs.insert(h->seg_graphs.begin(), es_graph_entry{key, exec});
  }
  if ((e = cudaGraphLaunch(exec, stream)) != cudaSuccess) return es_cuda_fail(h, e, "cudaGraphLaunch");
  return EXACTSUM_OK;
}

}  // namespace

void es_segment_free_extra(exactsum_t h) {
  clear_graphs(h);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  h->capture_stream = nullptr;
  cudaFree(h->seg_block_tiles);
  cudaFree(h->seg_tile_seg);
  h->seg_block_tiles = nullptr;
  h->seg_tile_seg = nullptr;
}

extern "C" {

exactsum_status exactsum_segmented_sum(exactsum_t h, const void* d_x, const int64_t* d_offsets,
                                       int64_t num_segments, exactsum_dtype in_dtype, exactsum_dtype out_dtype, exactsum_round mode,
                                       void* d_results, exactsum_stream_t stream) {
  exactsum_status st = check_seg_args(h, d_x, d_offsets, num_segments, in_dtype, out_dtype, mode, d_results);
  if (st != EXACTSUM_OK) return st;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return es_cuda_fail(h, e, "cudaSetDevice");
  if (num_segments == 0) return EXACTSUM_OK;
  return run_segmented(h, d_x, d_offsets, num_segments, in_dtype, out_dtype, mode, d_results,
                       (cudaStream_t)stream, lookup_config(h, in_dtype, num_segments), true);
}

exactsum_status exactsum_segmented_autotune(exactsum_t h, const void* d_x, const int64_t* d_offsets,
                                            int64_t num_segments, exactsum_dtype in_dtype, void* d_results_scratch,
                                            exactsum_stream_t stream, int* best_warps, int* best_kind,
                                            int64_t* best_tile, float* best_ms) {
  exactsum_status st =
      check_seg_args(h, d_x, d_offsets, num_segments, in_dtype, in_dtype, EXACTSUM_RNE, d_results_scratch);
  if (st != EXACTSUM_OK) return st;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return es_cuda_fail(h, e, "cudaSetDevice");
  if (num_segments == 0) return EXACTSUM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  es_seg_config best{};
  best.ms = -1.0f;
  const int64_t tiles_bytes[] = {64 << 10, 256 << 10, 1 << 20};
  // candidates: register form with either CTA size, and the TMA form
  const int forms[4][2] = {{0, es::SEG_KIND_REGISTER}, {1, es::SEG_KIND_REGISTER}, {2, es::SEG_KIND_TMA},
                           {3, es::SEG_KIND_WINDOW}};
  for (const auto& form : forms) {
    for (int64_t tb : tiles_bytes) {
      es_seg_config c;
      c.warps = es::seg_warps_choice(in_dtype, form[0]);
      c.kind = form[1];
      c.tile = tb / elem_bytes(in_dtype);
      c.ms = 0;
      // warm once, then time three calls
      st = run_segmented(h, d_x, d_offsets, num_segments, in_dtype, in_dtype, EXACTSUM_RNE,
                         d_results_scratch, s, c, false);
      if (st != EXACTSUM_OK) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3 && st == EXACTSUM_OK; ++r)
        st = run_segmented(h, d_x, d_offsets, num_segments, in_dtype, in_dtype, EXACTSUM_RNE,
                           d_results_scratch, s, c, false);
      cudaEventRecord(e1, s);
      if (st != EXACTSUM_OK) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
        st = es_cuda_fail(h, e, "autotune timing");
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      c.ms = ms / 3.0f;
      if (best.ms < 0 || c.ms < best.ms) best = c;
    }
    if (st != EXACTSUM_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != EXACTSUM_OK) return st;
  h->seg_tuning[in_dtype * 64 + ceil_log2(num_segments)] = best;
  if (best_warps) *best_warps = best.warps;
  if (best_kind) *best_kind = best.kind;
  if (best_tile) *best_tile = best.tile;
  if (best_ms) *best_ms = best.ms;
  return EXACTSUM_OK;
}

exactsum_status exactsum_tuning_save(exactsum_t h, const char* path) {
  if (!h || !path) return fail(h, EXACTSUM_EINVAL, "null handle or path");
  std::ofstream f(path);
  if (!f) return fail(h, EXACTSUM_EINVAL, std::string("cannot write ") + path);
  f << "{\"segmented\": [";
  bool first = true;
  for (const auto& kv : h->seg_tuning) {
    f << (first ? "" : ", ") << "{\"in_dtype\": " << kv.first / 64 << ", \"log2_segments\": " << kv.first % 64
      << ", \"warps\": " << kv.second.warps << ", \"kind\": " << kv.second.kind << ", \"tile\": "
      << kv.second.tile << ", \"ms\": " << kv.second.ms
      << "}";
    first = false;
  }
  f << "]}\n";
  return f.good() ? EXACTSUM_OK : fail(h, EXACTSUM_EINVAL, "write failed");
}

exactsum_status exactsum_tuning_load(exactsum_t h, const char* path) {
  if (!h || !path) return fail(h, EXACTSUM_EINVAL, "null handle or path");
  std::ifstream f(path);
  if (!f) return fail(h, EXACTSUM_EINVAL, std::string("cannot read ") + path);
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string text = ss.str();
  // entries are flat objects with the four integer fields written by save()
  size_t pos = 0;
  int loaded = 0;
  while ((pos = text.find('{', pos + 1)) != std::string::npos) {
    const size_t end = text.find('}', pos);
    if (end == std::string::npos) break;
    const std::string obj = text.substr(pos, end - pos);
    auto field = [&](const char* name, long long& v) {
      const size_t k = obj.find(std::string("\"") + name + "\"");
      if (k == std::string::npos) return false;
      const size_t c = obj.find(':', k);
      if (c == std::string::npos) return false;
      v = std::atoll(obj.c_str() + c + 1);
      return true;
    };
    long long in = 0, lg = 0, w = 0, tile = 0, kind = 0;
    if (field("in_dtype", in) && field("log2_segments", lg) && field("warps", w) && field("tile", tile)) {
      field("kind", kind);  // absent in older files: register form
      const bool in_ok = in >= 0 && in <= 2;
      const bool shape_ok =
          kind == es::SEG_KIND_TMA      ? (in_ok && w == es::seg_warps_choice((int)in, 2))
          : kind == es::SEG_KIND_WINDOW ? (in_ok && w == es::seg_warps_choice((int)in, 3))
                                        : (kind == es::SEG_KIND_REGISTER && in_ok &&
                                           (w == es::seg_warps_choice((int)in, 0) ||
                                            w == es::seg_warps_choice((int)in, 1)));
      if (in < 0 || in > 2 || lg < 0 || lg > 62 || tile <= 0 || !shape_ok)
        return fail(h, EXACTSUM_EINVAL, "invalid tuning entry");
      es_seg_config c;
      c.warps = (int)w;
      c.kind = (int)kind;
      c.tile = tile;
      c.ms = -1.0f;
      h->seg_tuning[(int)in * 64 + (int)lg] = c;
      ++loaded;
    }
    pos = end;
  }
  return loaded >= 0 ? EXACTSUM_OK : EXACTSUM_EINVAL;
}

exactsum_status exactsum_device_status(exactsum_t h, int64_t* status_out) {
  if (!h || !status_out) return fail(h, EXACTSUM_EINVAL, "null handle or output");
  *status_out = 0;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return es_cuda_fail(h, e, "cudaSetDevice");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return es_cuda_fail(h, e, "cudaDeviceSynchronize");
  unsigned long long v = 0;
  if ((e = cudaMemcpy(&v, h->dev_status, sizeof v, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaMemcpy(status)");
  const unsigned long long zero = 0;
  if ((e = cudaMemcpy(h->dev_status, &zero, sizeof zero, cudaMemcpyHostToDevice)) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaMemcpy(status)");
  *status_out = (int64_t)v;
  return EXACTSUM_OK;
}

exactsum_status exactsum_sum_each(exactsum_t h, const void* d_x, const int64_t* h_offsets, int64_t num_segments,
                                  exactsum_dtype in_dtype, exactsum_dtype out_dtype, exactsum_round mode, void* d_results,
                                  exactsum_stream_t stream) {
  exactsum_status st = check_seg_args(h, d_x, h_offsets, num_segments, in_dtype, out_dtype, mode, d_results);
  if (st != EXACTSUM_OK) return st;
  for (int64_t s = 0; s < num_segments; ++s)
    if (h_offsets[s] < 0 || h_offsets[s + 1] < h_offsets[s])
      return fail(h, EXACTSUM_EINVAL, "offsets must be non-negative and non-decreasing");
  const int eb = elem_bytes(in_dtype), ob = elem_bytes(out_dtype);
  for (int64_t s = 0; s < num_segments; ++s) {
    st = exactsum_sum(h, (const char*)d_x + (size_t)h_offsets[s] * eb, h_offsets[s + 1] - h_offsets[s], in_dtype,
                      out_dtype, mode, (char*)d_results + (size_t)s * ob, stream);
    if (st != EXACTSUM_OK) return st;
  }
  return EXACTSUM_OK;
}

}  // extern "C"
