// workspace.cu -- handle workspace and the host-buffer (end-to-end) pipeline.
#include <cuda_runtime.h>

#include <cstring>

#include "digits.cuh"
#include "handle.h"

exactsum_status es_workspace_init(exactsum_t h) {
  cudaError_t e;
  h->partial_rows = 2 * h->num_sms;
  if ((e = cudaMalloc(&h->partials, (size_t)h->partial_rows * es::ACC_WORDS * sizeof(int64_t))) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaMalloc(partials)");
  if ((e = cudaMalloc(&h->ticket, 64)) != cudaSuccess) return es_cuda_fail(h, e, "cudaMalloc(ticket)");
  if ((e = cudaMemset(h->ticket, 0, 64)) != cudaSuccess) return es_cuda_fail(h, e, "cudaMemset(ticket)");
  if ((e = cudaMalloc(&h->dev_status, 64)) != cudaSuccess) return es_cuda_fail(h, e, "cudaMalloc(status)");
  if ((e = cudaMemset(h->dev_status, 0, 64)) != cudaSuccess) return es_cuda_fail(h, e, "cudaMemset(status)");
  if ((e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaStreamCreate");
  for (int i = 0; i < 2; ++i) {
    if ((e = cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming)) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaEventCreate");
    if ((e = cudaEventCreateWithFlags(&h->ev_consumed[i], cudaEventDisableTiming)) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaEventCreate");
  }
  if ((e = cudaMalloc(&h->host_acc, es::ACC_WORDS * sizeof(int64_t))) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaMalloc(acc)");
  if ((e = cudaMalloc(&h->d_result_tmp, 64)) != cudaSuccess) return es_cuda_fail(h, e, "cudaMalloc(result)");
  if ((e = cudaMallocHost(&h->h_result_pinned, 64)) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaMallocHost(result)");
  return EXACTSUM_OK;
}

void es_workspace_free(exactsum_t h) {
  cudaFree(h->partials);
  cudaFree(h->ticket);
  cudaFree(h->dev_status);
  for (int i = 0; i < 2; ++i) {
    if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
    if (h->ev_consumed[i]) cudaEventDestroy(h->ev_consumed[i]);
    cudaFree(h->stage[i]);
  }
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  cudaFree(h->host_acc);
  cudaFree(h->d_result_tmp);
  if (h->h_result_pinned) cudaFreeHost(h->h_result_pinned);
  cudaFree(h->trunc_state);
  if (h->trunc_state_host) cudaFreeHost(h->trunc_state_host);
  es_segment_free_extra(h);
  cudaFree(h->seg_acc);
  cudaFree(h->seg_tile_base);
  cudaFree(h->seg_remaining);
  cudaFree(h->seg_counters);
  h->partials = nullptr;
}

// Host-resident input: copy it in chunks on the handle's copy stream while
// the previous chunk is added into a device accumulator on `stream`
// (double buffered), then round the accumulator and bring the result back.
// This is the external-memory scan of Section 5 (Theorem 5) with host
// memory as the external memory: one pass over the input, the accumulator
// resident on the device throughout.
exactsum_status es_sum_host_pipelined(exactsum_t h, const void* h_x, int64_t n, int in, int out,
                                      int mode, void* h_result, cudaStream_t stream) {
  const size_t kStage = (size_t)64 << 20;
  cudaError_t e;
  if (!h->stage[0]) {
    for (int i = 0; i < 2; ++i)
      if ((e = cudaMalloc(&h->stage[i], kStage)) != cudaSuccess) return es_cuda_fail(h, e, "cudaMalloc(stage)");
    h->stage_bytes = kStage;
  }
  const int eb = in == 0 ? 8 : (in == 1 ? 4 : 2);
  const int64_t chunk = (int64_t)(h->stage_bytes / eb);
  if ((e = cudaMemsetAsync(h->host_acc, 0, es::ACC_WORDS * sizeof(int64_t), stream)) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaMemsetAsync(acc)");
  int k = 0;
  for (int64_t off = 0; off < n; off += chunk, ++k) {
    const int b = k & 1;
    const int64_t cnt = (n - off < chunk) ? (n - off) : chunk;
    if ((e = cudaStreamWaitEvent(h->copy_stream, h->ev_consumed[b], 0)) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaStreamWaitEvent");
    if ((e = cudaMemcpyAsync(h->stage[b], (const char*)h_x + (size_t)off * eb, (size_t)cnt * eb,
                             cudaMemcpyHostToDevice, h->copy_stream)) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaMemcpyAsync(H2D)");
    if ((e = cudaEventRecord(h->ev_copied[b], h->copy_stream)) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(stream, h->ev_copied[b], 0)) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaStreamWaitEvent");
    es::SumArgs a = es_make_sum_args(h->stage[b], cnt, in);
    a.out = in;
    a.mode = 0;
    a.result = nullptr;
    a.acc = h->host_acc;
    a.partials = h->partials;
    a.ticket = h->ticket;
    a.status = h->dev_status;
    if ((e = es::launch_sum(in, a, h->max_ctas, stream, nullptr)) != cudaSuccess)
      return es_cuda_fail(h, e, "accumulate kernel launch");
    if ((e = cudaEventRecord(h->ev_consumed[b], stream)) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaEventRecord");
  }
  if ((e = es::launch_round_acc(h->host_acc, in, out, mode, h->d_result_tmp, stream)) != cudaSuccess)
    return es_cuda_fail(h, e, "round kernel launch");
  const int ob = out == 0 ? 8 : (out == 1 ? 4 : 2);
  if ((e = cudaMemcpyAsync(h->h_result_pinned, h->d_result_tmp, ob, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaMemcpyAsync(D2H)");
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return es_cuda_fail(h, e, "cudaStreamSynchronize");
  std::memcpy(h_result, h->h_result_pinned, ob);
  return EXACTSUM_OK;
}

exactsum_status es_segment_workspace_reserve(exactsum_t h, int64_t segments) {
  if (segments <= h->seg_capacity) return EXACTSUM_OK;
  cudaError_t e;
  cudaFree(h->seg_acc);
  cudaFree(h->seg_tile_base);
  cudaFree(h->seg_remaining);
  h->seg_acc = nullptr;
  h->seg_tile_base = nullptr;
  h->seg_remaining = nullptr;
  h->seg_capacity = 0;
  if ((e = cudaMalloc(&h->seg_acc, (size_t)segments * es::ACC_WORDS * sizeof(int64_t))) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaMalloc(segment accumulators)");
  if ((e = cudaMemset(h->seg_acc, 0, (size_t)segments * es::ACC_WORDS * sizeof(int64_t))) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaMemset(segment accumulators)");
  if ((e = cudaMalloc(&h->seg_tile_base, (size_t)(segments + 1) * sizeof(int64_t))) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaMalloc(tile bases)");
  if ((e = cudaMalloc(&h->seg_remaining, (size_t)segments * sizeof(unsigned int))) != cudaSuccess)
    return es_cuda_fail(h, e, "cudaMalloc(tile counters)");
  if (!h->seg_counters) {
    if ((e = cudaMalloc(&h->seg_counters, 64 * sizeof(unsigned long long))) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaMalloc(counters)");
    if ((e = cudaMemset(h->seg_counters, 0, 64 * sizeof(unsigned long long))) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaMemset(counters)");
  }
  h->seg_capacity = segments;
  return EXACTSUM_OK;
}
