// internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace es {

// Arguments of the single-array sum kernel.
struct SumArgs {
  const void* x;       // input (element-aligned)
  int64_t n;           // elements
  int64_t head;        // elements before the first 16-byte boundary (CTA 0)
  int64_t nvec;        // 16-byte vectors after the head
  int64_t tail;        // elements after the vectors (last CTA)
  int out, mode;       // output format and rounding mode
  void* result;        // result element (result mode)
  int64_t* acc;        // accumulator to add into (accumulate mode), or null
  int64_t* partials;   // grid x ACC_WORDS scratch
  unsigned int* ticket;  // zero between launches; reset by the last CTA
  unsigned long long* status;  // device status word (STATUS_* bits)
};

// Device status bits (also in include/exactsum.h as EXACTSUM_STATUS_*).
constexpr unsigned long long STATUS_BAD_OFFSETS = 1ull, STATUS_MAP_OVERFLOW = 2ull, STATUS_TIMEOUT = 4ull;

cudaError_t launch_sum(int in_dt, const SumArgs& a, int max_ctas, cudaStream_t stream, int* grid_out);
cudaError_t preload_sum_kernels();
// BF16 single-array kernels on FP32 digit columns (sum_bf16.cu); launch =
// false only loads and configures the kernel.
cudaError_t launch_sum_bf16(const SumArgs& a, int max_ctas, cudaStream_t stream, int* grid_out, bool launch);
cudaError_t trunc_preload();
cudaError_t launch_round_acc(const int64_t* acc, int in_dt, int out, int mode, void* result,
                             cudaStream_t stream);

}  // namespace es
