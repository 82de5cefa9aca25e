// sum_kernels.cu -- single-array exact sum (the hot path).
//
// Structure (Section 5, Theorem 5: when the accumulator fits in internal
// memory, keep it there and stream the input once, adding components in any
// order; Section 6.1: each reducer produces one accumulator and a final
// post-process adds the p accumulators and rounds):
//
//   1. every thread owns a private superaccumulator in shared memory
//      (digit-major, thread-minor layout: no bank conflicts for any digit
//      pattern) and adds the elements of its share of the array into it,
//      regularising every REG_EVERY additions (Lemma 1, deferred carries);
//   2. the CTA sums its threads' regularised digits (carry-free);
//   3. each CTA writes one 80-word partial accumulator; the last CTA to
//      finish (an atomic ticket, no waiting) sums the partials carry-free and
//      either rounds the result (Section 3 steps 6-7) or adds it into a
//      caller-held accumulator.
//
// One persistent CTA per SM; 16-byte read-only streaming loads, double
// buffered in registers so that each thread keeps two batches in flight.
#include <cuda_runtime.h>

#include "digits.cuh"
#include "finalize.cuh"
#include "internal.h"
#include "stream.cuh"

namespace es {

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

template <int DT, int T, int U>
__global__ void __launch_bounds__(T, 1) sum_kernel(SumArgs a) {
  constexpr int ND = Geometry<DT>::DIGITS;
  constexpr int REG_EVERY = Geometry<DT>::REG_EVERY;
  constexpr int NW = T / 32;
  static_assert(ND * T >= NW * ACC_WORDS, "digit area reused for the grid merge");

  extern __shared__ int64_t digits[];  // ND x T
  __shared__ int64_t blk[ACC_WORDS];
  __shared__ uint32_t limbs[ACC_DIGITS];
  __shared__ uint32_t blk_flags, is_last;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int64_t* col = digits + t;
#pragma unroll 4
  for (int i = 0; i < ND; ++i) col[i * T] = 0;
  if (t == 0) blk_flags = 0;

  uint32_t emax = 0;
  const uint4* vx = reinterpret_cast<const uint4*>((const char*)a.x + a.head * Geometry<DT>::ELEM_BYTES);
  const int64_t G = gridDim.x;
  const int64_t vb = a.nvec * blockIdx.x / G, ve = a.nvec * (blockIdx.x + 1) / G;
  int reg_left = REG_EVERY;

  // ---- hot loop: this thread's vectors vb + t + j*T, double buffered ----
  const int64_t cnt = (vb + t < ve) ? (ve - vb - t + T - 1) / T : 0;
  stream_add<DT, T, T, U>(col, vx + vb + t, cnt, emax, reg_left, t, vx + ve);

  // ---- unaligned head (CTA 0) and ragged tail (last CTA) ----
  if (blockIdx.x == 0 && t < a.head) add_one<DT, T>(col, load_one<DT>(a.x, t), emax);
  if (blockIdx.x == G - 1 && t < a.tail) add_one<DT, T>(col, load_one<DT>(a.x, a.n - a.tail + t), emax);
  regularise<DT, T>(col);

  // ---- special values and signed zeros: exact rescan only when needed ----
  uint32_t flags = 24u;  // an element with 0 < E < all-ones is neither +0 nor -0
  if (emax == Geometry<DT>::EXP_SPECIAL || emax == 0u) flags = rescan_flags<DT, T>(a, vb, ve);
  __syncthreads();
  if (flags) atomicOr(&blk_flags, flags);

  // ---- CTA merge: sum the threads' digits, carry-free ----
  for (int i = warp; i < ACC_DIGITS; i += NW) {
    int64_t s = 0;
    for (int j = lane; j < T; j += 32) s += digit32<DT, T>(digits + j, i);
    s = warp_sum(s);
    if (lane == 0) blk[i] = s;
  }
  __syncthreads();
  if (t < ACC_WORDS - ACC_DIGITS) {
    const int w = ACC_DIGITS + t;
    int64_t v = 0;
    if (w == W_NAN) v = (blk_flags & 1u) ? 1 : 0;
    else if (w == W_PINF) v = (blk_flags & 2u) ? 1 : 0;
    else if (w == W_NINF) v = (blk_flags & 4u) ? 1 : 0;
    else if (w == W_NOTPZ) v = (blk_flags & 8u) ? 1 : 0;
    else if (w == W_NOTNZ) v = (blk_flags & 16u) ? 1 : 0;
    else if (w == W_COUNT) v = (blockIdx.x == 0) ? a.n : 0;
    blk[w] = v;
  }
  __syncthreads();
  if (t < ACC_WORDS) a.partials[blockIdx.x * ACC_WORDS + t] = blk[t];
  __threadfence();
  __syncthreads();
  if (t == 0) is_last = (atomicAdd(a.ticket, 1u) == (unsigned)(G - 1)) ? 1u : 0u;
  __syncthreads();
  if (!is_last) return;

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

// Round a caller-held accumulator (one thread).
__global__ void round_acc_kernel(const int64_t* acc, int in_dt, int out, int mode, void* result) {
  __shared__ int64_t blk[ACC_WORDS];
  __shared__ uint32_t limbs[ACC_DIGITS];
  if (threadIdx.x == 0) {
    for (int w = 0; w < ACC_WORDS; ++w) blk[w] = acc[w];
    store_result(result, out, finalize_acc(blk, limbs, in_dt, out, mode));
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <int DT>
struct SumConfig;
#ifndef ES_F64_T
#define ES_F64_T 384
#endif
#ifndef ES_F64_U
#define ES_F64_U 4
#endif
#ifndef ES_F32_T
#define ES_F32_T 512
#endif
#ifndef ES_F32_U
#define ES_F32_U 4
#endif
#ifndef ES_BF16_T
#define ES_BF16_T 512
#endif
#ifndef ES_BF16_U
#define ES_BF16_U 2
#endif
template <> struct SumConfig<F64> { static constexpr int T = ES_F64_T, U = ES_F64_U; };
template <> struct SumConfig<F32> { static constexpr int T = ES_F32_T, U = ES_F32_U; };
template <> struct SumConfig<BF16> { static constexpr int T = ES_BF16_T, U = ES_BF16_U; };

template <int DT>
static cudaError_t launch_sum_t(const SumArgs& a0, int max_ctas, cudaStream_t stream, int* grid_out) {
  constexpr int T = SumConfig<DT>::T, U = SumConfig<DT>::U;
  constexpr size_t SMEM = (size_t)Geometry<DT>::DIGITS * T * sizeof(int64_t);
  static bool configured[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    e = cudaFuncSetAttribute(sum_kernel<DT, T, U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  SumArgs a = a0;
  // at least two vectors per thread per CTA, at most one CTA per SM
  int64_t want = (a.nvec + 2 * T - 1) / (2 * T);
  int grid = (int)(want < 1 ? 1 : (want > max_ctas ? max_ctas : want));
  if (grid_out) *grid_out = grid;
  sum_kernel<DT, T, U><<<grid, T, SMEM, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sum(int in_dt, const SumArgs& a, int max_ctas, cudaStream_t stream, int* grid_out) {
  switch (in_dt) {
    case F64: return launch_sum_t<F64>(a, max_ctas, stream, grid_out);
    case F32: return launch_sum_t<F32>(a, max_ctas, stream, grid_out);
    default: return launch_sum_t<BF16>(a, max_ctas, stream, grid_out);
  }
}

cudaError_t launch_round_acc(const int64_t* acc, int in_dt, int out, int mode, void* result,
                             cudaStream_t stream) {
  round_acc_kernel<<<1, 32, 0, stream>>>(acc, in_dt, out, mode, result);
  return cudaGetLastError();
}

int sum_threads_per_cta(int in_dt) {
  return in_dt == F64 ? SumConfig<F64>::T : (in_dt == F32 ? SumConfig<F32>::T : SumConfig<BF16>::T);
}

}  // namespace es
