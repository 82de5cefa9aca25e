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



// ---------------------------------------------------------------------------
// Resident express kernel (see serve.h).  Each CTA: SERVE_W - 1 worker warps
// and one poller warp (the last; its digit columns stay unused).  The poller reads the published tile count from pinned
// host memory every few hundred nanoseconds and keeps it in shared memory;
// workers claim tiles against that count.  Every wait is bounded: a CTA that
// has seen no new tile for idle_ns leaves (after a last look at the queue,
// see below), and the host launches the kernel again when it publishes work
// with no CTA alive.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ long long ld_relaxed_sys_s64(const void* p) {
  long long v;
  asm volatile("ld.relaxed.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_sys_s32(const void* p) {
  int v;
  asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_cta_shared_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.cta.shared::cta.u64 %0, [%1];" : "=l"(v) : "r"((uint32_t)__cvta_generic_to_shared(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cta_shared_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.cta.shared::cta.u64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "l"(v) : "memory");
}
__device__ __forceinline__ long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

// The descriptor of request q, read from the host ring with four 16-byte
// loads (one round trip to host memory).
__device__ __forceinline__ XDesc load_desc(const XDesc* d) {
  XDesc r;
  unsigned long long* w = reinterpret_cast<unsigned long long*>(&r);
  const unsigned long long* p = reinterpret_cast<const unsigned long long*>(d);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(w[2 * k]), "=l"(w[2 * k + 1]) : "l"(p + 2 * k)
                 : "memory");
  return r;
}

__global__ void __launch_bounds__(SERVE_T, 1) serve_resident_kernel(XArgs a) {
  extern __shared__ int64_t digits[];  // SERVE_ND x SERVE_T
  __shared__ int64_t wacc[SERVE_W][ACC_WORDS];
  __shared__ uint32_t wlimbs[SERVE_W][ACC_DIGITS];
  __shared__ unsigned long long s_req;  // published requests, as last seen by the poller
  __shared__ int s_exit;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int i = 0; i < SERVE_ND; ++i) digits[i * SERVE_T + t] = 0;
  if (t == 0) {
    s_req = ld_acquire_sys_u64(&a.q->tail_req);
    s_exit = 0;
  }
  __syncthreads();

  if (warp == SERVE_W - 1) {
    // ---- poller ----
    if (lane == 0) {
      unsigned long long seen = s_req;
      long long last_new = global_ns();
      for (;;) {
        const unsigned long long tl = ld_acquire_sys_u64(&a.q->tail_req);
        const long long now = global_ns();
        if (tl != seen) {
          seen = tl;
          st_release_cta_shared_u64(&s_req, tl);
          last_new = now;
        }
        const int stop = ld_relaxed_sys_s32(&a.q->stop);
        if (stop || now - last_new > a.idle_ns) {
          // leave the alive count, then look at the queue once more: either
          // this look sees a request the host published meanwhile (and the
          // CTA stays), or the host's look at the alive count, made after
          // its publication, sees this CTA gone and launches the kernel again
          atomicSub_system(&a.q->alive, 1);
          __threadfence_system();
          const unsigned long long tl2 = ld_acquire_sys_u64(&a.q->tail_req);
          if (tl2 != seen && !stop) {
            atomicAdd_system(&a.q->alive, 1);
            seen = tl2;
            st_release_cta_shared_u64(&s_req, tl2);
            last_new = global_ns();
            continue;
          }
          *(volatile int*)&s_exit = 1;
          break;
        }
        __nanosleep(256);
      }
    }
    return;
  }

  // ---- workers: requests in ring order, tiles claimed per request ----
  int64_t* col = digits + t;
  int64_t* warp_cols = digits + warp * 32;
  long long r = a.first_req;  // the request this warp takes tiles from
  XDesc d;
  bool have = false;
  for (;;) {
    const long long R = (long long)ld_acquire_cta_shared_u64(&s_req);
    if (r >= R) {
      if (*(volatile int*)&s_exit) break;
      __nanosleep(128);
      continue;
    }
    if (R > XRING && r < R - XRING) {  // far behind: those requests are complete
      r = R - XRING;
      have = false;
    }
    if (!have) {
      d = load_desc(&a.q->ring[r & (XRING - 1)]);
      if (d.q != r) {  // an entry already reused: that request is complete
        ++r;
        continue;
      }
      have = true;
    }
    // claim the next tile of request r.  The counter's high word is the
    // index (mod 2^32) of the request it counts for; requests at one ring
    // position differ by multiples of XRING and are compared as serial
    // numbers: an older one is replaced (its request is complete: the host
    // reuses a position only then), a newer one means request r is complete.
    unsigned long long* ctr = a.tiles + (r & (XRING - 1));
    long long k = -1;
    if (lane == 0) {
      const uint32_t g = (uint32_t)r;
      const unsigned long long tag = (unsigned long long)g << 32;
      unsigned long long v = *(volatile unsigned long long*)ctr;
      while ((int32_t)((uint32_t)(v >> 32) - g) < 0) {
        const unsigned long long old = atomicCAS(ctr, v, tag);
        v = (old == v) ? tag : old;
      }
      if ((v >> 32) == g && (long long)(v & 0xFFFFFFFFull) < d.ntiles) {
        const unsigned long long got = atomicAdd(ctr, 1ull);
        if ((got >> 32) == g && (long long)(got & 0xFFFFFFFFull) < d.ntiles) k = (long long)(got & 0xFFFFFFFFull);
      }
    }
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k < 0) {  // request r has no tile left: the next one
      ++r;
      have = false;
      continue;
    }
    const int64_t lo = k * d.tile;
    const int64_t hi = min((int64_t)d.n, (int64_t)(lo + d.tile));
    int64_t d0, d1, d2;
    uint32_t flags = 0;
    if (d.in == F64) serve_tile<F64>(col, warp_cols, d.x, lo, hi, lane, d0, d1, d2, flags);
    else if (d.in == F32) serve_tile<F32>(col, warp_cols, d.x, lo, hi, lane, d0, d1, d2, flags);
    else serve_tile<BF16>(col, warp_cols, d.x, lo, hi, lane, d0, d1, d2, flags);
    if (lane + 64 >= ACC_DIGITS) d2 = (lane + 64 < ACC_WORDS) ? flag_word(lane + 64, flags, hi - lo) : 0;
    unsigned long long* acc = (unsigned long long*)(a.slot_acc + (int64_t)d.slot * ACC_WORDS);
    if (d0) atomicAdd(acc + lane, (unsigned long long)d0);
    if (d1) atomicAdd(acc + lane + 32, (unsigned long long)d1);
    if (lane + 64 < ACC_WORDS && d2) atomicAdd(acc + lane + 64, (unsigned long long)d2);
    __threadfence();
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) last = (atomicAdd(a.done + d.slot, 1u) == (unsigned)(d.ntiles - 1)) ? 1u : 0u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      wacc[warp][lane] = (int64_t)__ldcg(acc + lane);
      wacc[warp][lane + 32] = (int64_t)__ldcg(acc + lane + 32);
      if (lane + 64 < ACC_WORDS) wacc[warp][lane + 64] = (int64_t)__ldcg(acc + lane + 64);
      // the slot starts its next request from zero
      acc[lane] = 0;
      acc[lane + 32] = 0;
      if (lane + 64 < ACC_WORDS) acc[lane + 64] = 0;
      if (lane == 0) a.done[d.slot] = 0u;
      __syncwarp();
      if (lane == 0) {
        const uint64_t bits = finalize_acc(wacc[warp], wlimbs[warp], d.in, d.out, d.mode);
        volatile ServeDone* res = a.results + d.slot;
        res->bits = bits;
        __threadfence_system();
        res->seq = (unsigned long long)r + 1ull;
      }
      __syncwarp();
    }
  }
}

cudaError_t serve_resident_configure() {
  return cudaFuncSetAttribute(serve_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(SERVE_ND * SERVE_T * sizeof(int64_t)));
}

cudaError_t serve_resident_launch(const XArgs& a, int grid, cudaStream_t stream) {
  serve_resident_kernel<<<grid, SERVE_T, SERVE_ND * SERVE_T * sizeof(int64_t), stream>>>(a);
  return cudaGetLastError();
}
}  // namespace es
