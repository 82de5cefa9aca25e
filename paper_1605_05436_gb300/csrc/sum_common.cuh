// sum_common.cuh -- the parts of the single-array sum kernels that every
// input format shares: the exact rescan for special values and signed
// zeros, the CTA merge and the last-CTA grid merge (Section 6.1: each
// reducer writes one partial accumulator, a post-process adds them and
// rounds once), and the one-time kernel set-up.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include "digits.cuh"
#include "finalize.cuh"
#include "internal.h"
#include "stream.cuh"

// BF16 single-array kernel: 2 the FP32-digit kernel fed by a TMA ring
// (sum_bf16.cu), 1 its register-loading form, 0 the integer digit columns
// (sum_kernels.cu).
#ifndef ES_BF16_FFMA
#define ES_BF16_FFMA 2
#endif

namespace es {

// Programmatic dependent launch of the single-array kernels: a launch may start streaming
// while the one before it on the stream merges and rounds (it waits for that
// one before it touches the shared partials, ticket or result).  Only a
// kernel that signals its dependents (this one) lets the next launch start
// early; after any other stream operation the launch waits as usual.
// (Back to back at 2^28: 0.3572 ms per launch against 0.3590 without.)
#ifndef ES_PDL
#define ES_PDL 1
#endif
// Vectors the last CTA of a single-array kernel gives up to the others.  Back to back,
// the SM whose CTA merges and rounds frees up last, so the next launch's
// last CTA (dispatched last) starts there about 8 us late; with that much
// less to stream (about 19,000 vectors at the per-SM rate) it finishes with
// the others.  With the launches serialised it is off the critical path.
// (Back to back at 2^28: 0.3511 ms per launch against 0.3584; 38,912: 0.3500.)
#ifndef ES_TAIL_CUT
#define ES_TAIL_CUT 19456
#endif

// The two halves of programmatic dependent launch inside a kernel: let the
// next launch on the stream start as this one's CTAs leave, and wait for the
// launch before this one before touching the workspace it shared.
__device__ __forceinline__ void pdl_signal() {
#if ES_PDL
  asm volatile("griddepcontrol.launch_dependents;");
#endif
}
__device__ __forceinline__ void pdl_wait() {
#if ES_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

// This CTA's vectors [vb, ve) of nvec: equal shares, except that the last
// CTA gives up ES_TAIL_CUT vectors (at most a quarter of a share).
__device__ __forceinline__ void cta_range(int64_t nvec, int64_t& vb, int64_t& ve) {
  const int64_t G = gridDim.x;
#if ES_TAIL_CUT > 0
  const int64_t cut = min((int64_t)ES_TAIL_CUT, nvec / (4 * G));
  vb = (nvec + cut) * blockIdx.x / G;
  ve = blockIdx.x == G - 1 ? nvec : (nvec + cut) * (blockIdx.x + 1) / G;
#else
  vb = nvec * blockIdx.x / G;
  ve = nvec * (blockIdx.x + 1) / G;
#endif
}

// Launch a single-array kernel (with the programmatic-serialisation
// attribute when ES_PDL is set).
template <typename K>
static inline cudaError_t launch_single_array(K kernel, int grid, int threads, size_t smem, cudaStream_t stream,
                                              const SumArgs& a) {
#if ES_PDL
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, a);
#else
  kernel<<<grid, threads, smem, stream>>>(a);
  return cudaGetLastError();
#endif
}

// Elements owned by thread t of CTA b: vectors vb + t + j*T (< ve), the
// unaligned head (CTA 0) and the ragged tail (last CTA).
template <int DT, int T>
__device__ uint32_t rescan_flags(const SumArgs& a, int64_t vb, int64_t ve) {
  constexpr int EB = Geometry<DT>::ELEM_BYTES;
  constexpr int EPV = 16 / EB;
  const int t = threadIdx.x;
  uint32_t f = 0;
  const char* base = (const char*)a.x + a.head * EB;
  for (int64_t v = vb + t; v < ve; v += T)
    for (int e = 0; e < EPV; ++e) f |= classify<DT>(load_one<DT>(base, v * EPV + e));
  if (blockIdx.x == 0 && t < a.head) f |= classify<DT>(load_one<DT>(a.x, t));
  if (blockIdx.x == gridDim.x - 1 && t < a.tail) f |= classify<DT>(load_one<DT>(a.x, a.n - a.tail + t));
  return f;
}

// CTA merge and grid merge, shared by both single-array kernels.  Called by
// every thread of the CTA after its flags are in blk_flags and a barrier.
// TC threads own digit columns (digit-major, stride TC); NW warps take part.
// HALF: the columns count in half units of the input format (the BF16
// FP32-digit columns, fdigits.cuh); their exact sum is even and is halved
// here, digit by digit, before it leaves the CTA.
// SCRATCH: bytes available at `cols` (reused for the grid merge).
template <int DT, int TC, int NW, typename D, bool HALF = false,
          size_t SCRATCH = (size_t)Geometry<DT>::DIGITS * TC * sizeof(D)>
__device__ __forceinline__ void finish_cta(const SumArgs& a, D* cols, int64_t* blk, uint32_t* limbs,
                                           uint32_t blk_flags, uint32_t* is_last) {
  static_assert(SCRATCH >= NW * ACC_WORDS * sizeof(int64_t), "digit area reused for the grid merge");
  int64_t* digits = reinterpret_cast<int64_t*>(cols);  // scratch once the columns are merged
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t G = gridDim.x;
  // ---- CTA merge: sum the columns' digits, carry-free ----
  for (int i = warp; i < ACC_DIGITS; i += NW) {
    int64_t s = 0;
    for (int j = lane; j < TC; j += 32) s += digit32<DT, TC>(cols + j, i);
    s = warp_sum(s);
    if (lane == 0) blk[i] = s;
  }
  if (t < ACC_WORDS - ACC_DIGITS)
    blk[ACC_DIGITS + t] = flag_word(ACC_DIGITS + t, blk_flags, blockIdx.x == 0 ? a.n : 0);
  __syncthreads();
  if constexpr (HALF) {
    // V = sum D_i 2^(32 i) is even, so D_0 is even and
    // V / 2 = sum ((D_i >> 1) + (D_(i+1) & 1) 2^31) 2^(32 i)
    int64_t v = 0, up = 0;
    if (t < ACC_DIGITS) {
      v = blk[t];
      up = (t + 1 < ACC_DIGITS) ? blk[t + 1] : 0;
    }
    __syncthreads();
    if (t < ACC_DIGITS) blk[t] = (v >> 1) + ((up & 1) << 31);
    __syncthreads();
  }
  if (t < ACC_WORDS) a.partials[blockIdx.x * ACC_WORDS + t] = blk[t];
  __threadfence();
  __syncthreads();
  if (t == 0) *is_last = (atomicAdd(a.ticket, 1u) == (unsigned)(G - 1)) ? 1u : 0u;
  __syncthreads();
  if (!*is_last) return;

  // ---- last CTA: merge the partial accumulators (post-process) ----
  __threadfence();
  int64_t s0 = 0, s1 = 0, s2 = 0;
  for (int64_t r = warp; r < G; r += NW) {
    const int64_t* row = a.partials + r * ACC_WORDS;
    s0 += __ldcg((const long long*)row + lane);
    s1 += __ldcg((const long long*)row + lane + 32);
    if (lane + 64 < ACC_WORDS) s2 += __ldcg((const long long*)row + lane + 64);
  }
  digits[warp * ACC_WORDS + lane] = s0;
  digits[warp * ACC_WORDS + lane + 32] = s1;
  if (lane + 64 < ACC_WORDS) digits[warp * ACC_WORDS + lane + 64] = s2;
  __syncthreads();
  if (t < ACC_WORDS) {
    int64_t s = 0;
    for (int w = 0; w < NW; ++w) s += digits[w * ACC_WORDS + t];
    if (a.acc) s += a.acc[t];
    blk[t] = s;
  }
  __syncthreads();
  if (t == 0) {
    *a.ticket = 0u;  // ready for the next launch on this workspace
    if (a.acc) {
      regularise72(blk);
      for (int w = 0; w < ACC_WORDS; ++w) a.acc[w] = blk[w];
    } else {
      store_result(a.result, a.out, finalize_acc(blk, limbs, DT, a.out, a.mode));
    }
  }
}

// Set the dynamic shared-memory limit of a kernel once per device.
static inline cudaError_t configure_once(const void* fn, size_t smem, std::atomic<bool>* done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64) done[dev].store(true, std::memory_order_release);
  return cudaSuccess;
}

}  // namespace es
