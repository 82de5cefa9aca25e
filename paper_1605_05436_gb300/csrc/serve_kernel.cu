// serve_kernel.cu -- one continuous-batching step of the serving engine.
//
// A step carries one chunk of every active request (mixed FP64/FP32/BF16).
// Chunks are cut into tiles; the persistent warps of the step kernel pull
// tiles, sum them into lane-private superaccumulators, merge them
// carry-free and add the 80-word partial into the request's slot
// accumulator with integer atomics (Lemma 1: digit-wise addition, order
// free).  The slot accumulator lives on the device for the whole life of
// the request, across steps (the reducer state of Section 6.1 kept on the
// device).  The warp that retires the last tile of a request's final chunk
// rounds the slot (Section 3 steps 6-7), clears it and publishes the result
// to the host at once (pinned memory, system-scope fence, then a sequence
// number), so that a request never waits for the other chunks of its step.
#include <cuda_runtime.h>

#include "digits.cuh"
#include "finalize.cuh"
#include "serve.h"
#include "stream.cuh"

namespace es {

constexpr int SERVE_W = SERVE_WARPS_PER_CTA;
constexpr int SERVE_T = SERVE_W * 32;
#ifndef ES_SERVE_U
#define ES_SERVE_U 6
#endif
constexpr int SERVE_U = ES_SERVE_U;
constexpr int SERVE_ND = Geometry<F64>::DIGITS;  // column height (FP64 is the tallest)

template <int DT>
__device__ __forceinline__ void serve_tile(int64_t* col, int64_t* warp_cols, const void* x, int64_t lo,
                                           int64_t hi, int lane, int64_t& d0, int64_t& d1, int64_t& d2,
                                           uint32_t& flags) {
  const RangeSplit r = split_range<DT>(x, lo, hi);
  uint32_t emax = 0;
  int reg_left = Geometry<DT>::REG_EVERY;
  add_split<DT, SERVE_T, 32, SERVE_U>(col, x, r, lane, emax, reg_left);
  regularise<DT, SERVE_T>(col);
  uint32_t f = 24u;
  if (emax == Geometry<DT>::EXP_SPECIAL || emax == 0u) f = rescan_split<DT, 32>(x, r, lane);
  flags = __reduce_or_sync(0xffffffffu, f);
  __syncwarp();
  warp_merge<DT, SERVE_T>(warp_cols, lane, d0, d1, d2);
  __syncwarp();
  for (int i = 0; i < Geometry<DT>::DIGITS; ++i) col[i * SERVE_T] = 0;
}

__global__ void __launch_bounds__(SERVE_T, 1) serve_step_kernel(ServeStep st) {
  extern __shared__ int64_t digits[];  // SERVE_ND x SERVE_T
  __shared__ int64_t wacc[SERVE_W][ACC_WORDS];
  __shared__ uint32_t wlimbs[SERVE_W][ACC_DIGITS];
  __shared__ int64_t sbase[SERVE_MAX_ITEMS + 1];

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int64_t* col = digits + t;
  for (int i = 0; i < SERVE_ND; ++i) col[i * SERVE_T] = 0;
  const int nitems = st.nitems;
  if (nitems <= 0) return;
  for (int i = t; i <= nitems; i += SERVE_T) sbase[i] = st.items[min(i, nitems - 1)].tile_base +
                                                        (i == nitems ? st.items[nitems - 1].ntiles : 0);
  __syncthreads();
  const int64_t total = sbase[nitems];

  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(st.queue, 1ull);
    const int64_t tile = (int64_t)__shfl_sync(0xffffffffu, tk, 0);
    if (tile >= total) break;
    // item of this tile: last item whose first tile is <= tile
    int lo_i = 0, hi_i = nitems - 1;
    while (lo_i < hi_i) {
      const int mid = (lo_i + hi_i + 1) >> 1;
      if (sbase[mid] <= tile) lo_i = mid;
      else hi_i = mid - 1;
    }
    const ServeItem it = st.items[lo_i];
    const int64_t lo = (tile - it.tile_base) * it.tile;
    const int64_t hi = min(it.len, lo + it.tile);
    int64_t d0, d1, d2;
    uint32_t flags = 0;
    int64_t* warp_cols = digits + warp * 32;
    if (it.in == F64) serve_tile<F64>(col, warp_cols, it.x, lo, hi, lane, d0, d1, d2, flags);
    else if (it.in == F32) serve_tile<F32>(col, warp_cols, it.x, lo, hi, lane, d0, d1, d2, flags);
    else serve_tile<BF16>(col, warp_cols, it.x, lo, hi, lane, d0, d1, d2, flags);
    if (lane + 64 >= ACC_DIGITS) d2 = (lane + 64 < ACC_WORDS) ? flag_word(lane + 64, flags, hi - lo) : 0;

    unsigned long long* acc = (unsigned long long*)(st.slot_acc + (int64_t)it.slot * ACC_WORDS);
    if (d0) atomicAdd(acc + lane, (unsigned long long)d0);
    if (d1) atomicAdd(acc + lane + 32, (unsigned long long)d1);
    if (lane + 64 < ACC_WORDS && d2) atomicAdd(acc + lane + 64, (unsigned long long)d2);
    __threadfence();
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) last = (atomicSub(st.remaining + lo_i, 1u) == 1u) ? 1u : 0u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last && it.final) {
      __threadfence();
      wacc[warp][lane] = (int64_t)__ldcg(acc + lane);
      wacc[warp][lane + 32] = (int64_t)__ldcg(acc + lane + 32);
      if (lane + 64 < ACC_WORDS) wacc[warp][lane + 64] = (int64_t)__ldcg(acc + lane + 64);
      acc[lane] = 0;
      acc[lane + 32] = 0;
      if (lane + 64 < ACC_WORDS) acc[lane + 64] = 0;
      __syncwarp();
      if (lane == 0) {
        const uint64_t bits = finalize_acc(wacc[warp], wlimbs[warp], it.in, it.out, it.mode);
        volatile ServeDone* d = st.done + lo_i;
        d->bits = bits;
        __threadfence_system();
        d->seq = st.seq;
      }
      __syncwarp();
    }
  }
}

cudaError_t serve_configure() {
  return cudaFuncSetAttribute(serve_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(SERVE_ND * SERVE_T * sizeof(int64_t)));
}

cudaError_t serve_launch(const ServeStep& st, int grid, cudaStream_t stream) {
  serve_step_kernel<<<grid, SERVE_T, SERVE_ND * SERVE_T * sizeof(int64_t), stream>>>(st);
  return cudaGetLastError();
}

}  // namespace es
