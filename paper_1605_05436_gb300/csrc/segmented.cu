// segmented.cu -- many exact sums of CSR segments in one persistent launch.
//
// The MapReduce shape of Section 6.1, inside one GPU: the input is cut into
// tiles (a segment of length L becomes ceil(L / TILE) tiles); every warp is
// a reducer that pulls tiles from a work queue, sums its tile into private
// superaccumulators and merges them carry-free (Lemma 1).  A tile that is a
// whole segment is rounded by its warp at once.  Otherwise the warp adds its
// 80-word partial into the segment's accumulator with integer atomics
// (digit-wise addition is the carry-free superaccumulator sum, so the order
// of arrival does not matter), and the warp that retires the segment's last
// tile rounds it (the post-process of Section 6.1) and clears the
// accumulator for the next call.  Nothing waits on anything: the last
// arriver does the work.
//
// Launch sequence (captured once into a CUDA graph per call signature):
//   seg_count_kernel   tiles per segment, summed per 1024-segment block
//   seg_scan_kernel    exclusive scan of the block sums (one CTA)
//   seg_base_kernel    per-segment first tile, tile->segment map, empty
//                      segments answered (+0), invalid offsets flagged
//   seg_sum_kernel     the persistent reducer kernel
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/exactsum.h"
#include "digits.cuh"
#include "finalize.cuh"
#include "handle.h"
#include "segmented.h"
#include "stream.cuh"
#include "tma.cuh"
#include "window.cuh"

namespace es {

constexpr int PLAN_T = 1024;

__device__ __forceinline__ void store_indexed(void* results, int out, int64_t s, uint64_t bits) {
  const int w = out == F64 ? 8 : (out == F32 ? 4 : 2);
  store_result((char*)results + s * w, out, bits);
}

// Round a segment's accumulator into its result slot (one thread), out of
// line: the windowed reducer's streaming loop runs at 80 registers or fewer
// (24-32 warps), and the rounding inlined beside it spills.
__device__ __noinline__ void round_segment(const SegArgs& a, int64_t s, const int64_t* acc, uint32_t* limbs,
                                           int in_dt) {
  store_indexed(a.results, a.out, s, finalize_acc(acc, limbs, in_dt, a.out, a.mode));
}

__device__ __forceinline__ uint64_t quiet_nan_bits(int out) {
  return out == F64 ? 0x7FF8000000000000ull : (out == F32 ? 0x7FC00000ull : 0x7FC0ull);
}

__device__ __forceinline__ int64_t seg_tiles(const int64_t* off, int64_t s, int64_t tile, bool& bad) {
  const int64_t a = off[s], b = off[s + 1];
  if (a < 0 || b < a) {
    bad = true;
    return 0;
  }
  return (b - a + tile - 1) / tile;
}

// Block-wide exclusive scan of one int64 per thread (PLAN_T threads).
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* warp_tot, int64_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int64_t w = (lane < PLAN_T / 32) ? warp_tot[lane] : 0;
    int64_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < PLAN_T / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
    if (lane == 31) warp_tot[32] = wi;
  }
  __syncthreads();
  total = warp_tot[32];
  const int64_t r = warp_tot[warp] + inc - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(PLAN_T) seg_count_kernel(SegArgs a) {
  __shared__ int64_t warp_tot[33];
  const int64_t s = (int64_t)blockIdx.x * PLAN_T + threadIdx.x;
  bool bad = false;
  const int64_t nt = (s < a.S) ? seg_tiles(a.off, s, a.tile, bad) : 0;
  int64_t total;
  block_exclusive_scan(nt, warp_tot, total);
  if (threadIdx.x == 0) a.block_tiles[blockIdx.x] = total;
}

__global__ void __launch_bounds__(PLAN_T) seg_scan_kernel(SegArgs a, int64_t nblocks) {
  __shared__ int64_t warp_tot[33];
  int64_t running = 0;
  for (int64_t base = 0; base < nblocks; base += PLAN_T) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = (i < nblocks) ? a.block_tiles[i] : 0;
    int64_t total;
    const int64_t ex = block_exclusive_scan(v, warp_tot, total);
    if (i < nblocks) a.block_tiles[i] = running + ex;
    running += total;
  }
  if (threadIdx.x == 0) {
    a.counters[CNT_QUEUE] = 0;
    a.counters[CNT_TOTAL] = (unsigned long long)running;
    if ((int64_t)running > a.map_capacity) atomicOr(a.status, STATUS_MAP_OVERFLOW);
  }
}

__global__ void __launch_bounds__(PLAN_T) seg_base_kernel(SegArgs a) {
  __shared__ int64_t warp_tot[33];
  const int64_t s = (int64_t)blockIdx.x * PLAN_T + threadIdx.x;
  bool bad = false;
  const int64_t nt = (s < a.S) ? seg_tiles(a.off, s, a.tile, bad) : 0;
  int64_t total;
  const int64_t ex = block_exclusive_scan(nt, warp_tot, total);
  const int64_t base = a.block_tiles[blockIdx.x] + ex;
  const bool fits = (int64_t)__ldcg((const unsigned long long*)&a.counters[CNT_TOTAL]) <= a.map_capacity;
  if (s < a.S) {
    a.tile_base[s] = base;
    a.remaining[s] = (unsigned)nt;
    if (s == a.S - 1) a.tile_base[a.S] = base + nt;
    if (nt == 0) store_indexed(a.results, a.out, s, bad ? quiet_nan_bits(a.out) : 0ull);
    if (fits)
      for (int64_t k = 0; k < nt; ++k) a.tile_seg[base + k] = (int32_t)s;
    else if (nt > 0)
      store_indexed(a.results, a.out, s, quiet_nan_bits(a.out));
    if (bad) atomicOr(a.status, STATUS_BAD_OFFSETS);
  }
}

// Per-tile work item of the reducers.
struct TileWork {
  int64_t s;       // segment
  int64_t ntiles;  // tiles of the segment
  int64_t lo, hi;  // element range of this tile
};

__device__ __forceinline__ TileWork tile_work(const SegArgs& a, int64_t tile) {
  TileWork w;
  w.s = a.tile_seg[tile];
  const int64_t tb = a.tile_base[w.s];
  w.ntiles = a.tile_base[w.s + 1] - tb;
  w.lo = a.off[w.s] + (tile - tb) * a.tile;
  w.hi = min(a.off[w.s + 1], w.lo + a.tile);
  return w;
}

// Emit a tile's 80-word warp partial (lane L holds words L, L + 32, L + 64):
// round the segment at once if this tile is the whole segment, else add it
// into the segment's accumulator; the warp that retires the last tile of the
// segment rounds it and clears the accumulator.
// OOL: round through round_segment (out of line) instead of inline.
template <int DT, int W, bool OOL = false>
__device__ __forceinline__ void seg_emit(const SegArgs& a, const TileWork& w, int64_t d0, int64_t d1, int64_t d2,
                                         int64_t (*wacc)[ACC_WORDS], uint32_t (*wlimbs)[ACC_DIGITS]) {
  auto round_into = [&](int64_t s) {
    if constexpr (OOL) round_segment(a, s, wacc[threadIdx.x >> 5], wlimbs[threadIdx.x >> 5], DT);
    else store_indexed(a.results, a.out, s, finalize_acc(wacc[threadIdx.x >> 5], wlimbs[threadIdx.x >> 5], DT, a.out, a.mode));
  };
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (w.ntiles == 1) {
    wacc[warp][lane] = d0;
    wacc[warp][lane + 32] = d1;
    if (lane + 64 < ACC_WORDS) wacc[warp][lane + 64] = d2;
    __syncwarp();
    if (lane == 0) round_into(w.s);
    __syncwarp();
  } else {
    unsigned long long* acc = (unsigned long long*)(a.seg_acc + w.s * ACC_WORDS);
    if (d0) atomicAdd(acc + lane, (unsigned long long)d0);
    if (d1) atomicAdd(acc + lane + 32, (unsigned long long)d1);
    if (lane + 64 < ACC_WORDS && d2) atomicAdd(acc + lane + 64, (unsigned long long)d2);
    __threadfence();
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) last = (atomicSub(&a.remaining[w.s], 1u) == 1u) ? 1u : 0u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      wacc[warp][lane] = (int64_t)__ldcg(acc + lane);
      wacc[warp][lane + 32] = (int64_t)__ldcg(acc + lane + 32);
      if (lane + 64 < ACC_WORDS) wacc[warp][lane + 64] = (int64_t)__ldcg(acc + lane + 64);
      acc[lane] = 0;
      acc[lane + 32] = 0;
      if (lane + 64 < ACC_WORDS) acc[lane + 64] = 0;
      __syncwarp();
      if (lane == 0) round_into(w.s);
      __syncwarp();
    }
  }
}

// After a tile has been added into the warp's columns: regularise, classify,
// merge the warp carry-free, clear the columns, and either round the segment
// (a one-tile segment) or add the partial into the segment's accumulator;
// the warp that retires the last tile rounds it and clears the accumulator.
template <int DT, int T, int W>
__device__ __forceinline__ void seg_finish_tile(const SegArgs& a, const TileWork& w, const RangeSplit& r,
                                                int64_t* digits, int64_t* col, int64_t (*wacc)[ACC_WORDS],
                                                uint32_t (*wlimbs)[ACC_DIGITS], uint32_t emax) {
  constexpr int ND = Geometry<DT>::DIGITS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  regularise<DT, T>(col);
  uint32_t flags = 24u;
  if (emax == Geometry<DT>::EXP_SPECIAL || emax == 0u) flags = rescan_split<DT, 32>(a.x, r, lane);
  flags = __reduce_or_sync(0xffffffffu, flags);
  __syncwarp();

  // ---- warp merge (carry-free), then clear the columns ----
  int64_t d0, d1, d2;
  warp_merge<DT, T>(digits + warp * 32, lane, d0, d1, d2);
  __syncwarp();
  for (int i = 0; i < ND; ++i) col[i * T] = 0;
  if (lane + 64 >= ACC_DIGITS) d2 = (lane + 64 < ACC_WORDS) ? flag_word(lane + 64, flags, w.hi - w.lo) : 0;

  seg_emit<DT, W>(a, w, d0, d1, d2, wacc, wlimbs);
}

// Register-streaming reducer: each lane loads its own vectors.
template <int DT, int W, int U>
__global__ void __launch_bounds__(W * 32, 1) seg_sum_kernel(SegArgs a) {
  constexpr int T = W * 32;
  constexpr int ND = Geometry<DT>::DIGITS;
  constexpr int REG_EVERY = Geometry<DT>::REG_EVERY;
  extern __shared__ int64_t digits[];  // ND x T
  __shared__ int64_t wacc[W][ACC_WORDS];
  __shared__ uint32_t wlimbs[W][ACC_DIGITS];

  const int t = threadIdx.x, lane = t & 31;
  int64_t* col = digits + t;
  for (int i = 0; i < ND; ++i) col[i * T] = 0;
  const int64_t total = (int64_t)__ldcg((const unsigned long long*)&a.counters[CNT_TOTAL]);
  if (total > a.map_capacity) return;  // flagged by the planner; results are NaN

  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(&a.counters[CNT_QUEUE], 1ull);
    const int64_t tile = (int64_t)__shfl_sync(0xffffffffu, tk, 0);
    if (tile >= total) break;
    const TileWork w = tile_work(a, tile);
    const RangeSplit r = split_range<DT>(a.x, w.lo, w.hi);
    uint32_t emax = 0;
    int reg_left = REG_EVERY;
    add_split<DT, T, 32, U>(col, a.x, r, lane, emax, reg_left);
    seg_finish_tile<DT, T, W>(a, w, r, digits, col, wacc, wlimbs, emax);
  }
}

// TMA reducer: each warp streams its own tile through an S-stage ring in
// shared memory; lane 0 issues the bulk copies (cp.async.bulk) S batches
// ahead and refills a stage as soon as the warp has copied it to registers.
// Every wait is bounded; a timeout sets STATUS_TIMEOUT, waits (bounded) for
// the warp's copies still in flight and retires the warp.
template <int DT, int W, int U, int S>
__global__ void __launch_bounds__(W * 32, 1) seg_sum_kernel_tma(SegArgs a) {
  constexpr int T = W * 32;
  constexpr int ND = Geometry<DT>::DIGITS;
  constexpr int EB = Geometry<DT>::ELEM_BYTES;
  constexpr int EPV = 16 / EB;
  constexpr int REG_EVERY = Geometry<DT>::REG_EVERY;
  constexpr int B = 32 * U;  // vectors per batch of one warp
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int64_t* digits = reinterpret_cast<int64_t*>(smem_raw);                      // ND x T
  uint4* rings = reinterpret_cast<uint4*>(smem_raw + (size_t)ND * T * 8);      // W x S x B
  uint64_t* bars = reinterpret_cast<uint64_t*>(rings + (size_t)W * S * B);     // W x S
  __shared__ int64_t wacc[W][ACC_WORDS];
  __shared__ uint32_t wlimbs[W][ACC_DIGITS];

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int64_t* col = digits + t;
  for (int i = 0; i < ND; ++i) col[i * T] = 0;
  uint4* ring = rings + (size_t)warp * S * B;
  uint64_t* full = bars + warp * S;
  if (lane == 0) {
    for (int k = 0; k < S; ++k) mbar_init(&full[k], 1);
    mbar_init_fence();
  }
  __syncwarp();
  const int64_t total = (int64_t)__ldcg((const unsigned long long*)&a.counters[CNT_TOTAL]);
  if (total > a.map_capacity) return;  // flagged by the planner; results are NaN

  uint32_t g = 0;  // batches this warp has consumed: stage g % S, phase parity (g / S) & 1
  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(&a.counters[CNT_QUEUE], 1ull);
    const int64_t tile = (int64_t)__shfl_sync(0xffffffffu, tk, 0);
    if (tile >= total) break;
    const TileWork w = tile_work(a, tile);
    const RangeSplit r = split_range<DT>(a.x, w.lo, w.hi);
    uint32_t emax = 0;
    int reg_left = REG_EVERY;
    if (lane < r.head_n) add_one<DT, T>(col, load_one<DT>(a.x, r.vlo - r.head_n + lane), emax);
    const uint4* vp = reinterpret_cast<const uint4*>((const char*)a.x + r.vlo * EB);
    const int64_t nb = (r.nvec + B - 1) / B;
    if (lane == 0) {
      for (int64_t k = 0; k < nb && k < S; ++k) {
        const uint32_t st = (g + (uint32_t)k) % S;
        const int64_t nv = min((int64_t)B, r.nvec - k * B);
        mbar_arrive_expect_tx(&full[st], (uint32_t)(nv * 16));
        bulk_copy_g2s(ring + (size_t)st * B, vp + k * B, (uint32_t)(nv * 16), &full[st]);
      }
    }
    bool ok = true;
    int64_t k = 0;
    for (; k < nb; ++k) {
      const uint32_t gk = g + (uint32_t)k;
      const uint32_t st = gk % S;
      ok = mbar_wait(&full[st], (gk / S) & 1u);
      if (__any_sync(0xffffffffu, !ok)) {
        ok = false;
        break;
      }
      const int64_t nv = min((int64_t)B, r.nvec - k * B);
      const uint4* stage = ring + (size_t)st * B;
      uint4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (lane + 32 * u < nv) v[u] = lds128(stage + lane + 32 * u);
      __syncwarp();
      if (lane == 0 && k + S < nb) {
        // the warp's reads of this stage are done: order them before the
        // asynchronous refill of the same stage
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const int64_t nv2 = min((int64_t)B, r.nvec - (k + S) * B);
        mbar_arrive_expect_tx(&full[st], (uint32_t)(nv2 * 16));
        bulk_copy_g2s(ring + (size_t)st * B, vp + (k + S) * B, (uint32_t)(nv2 * 16), &full[st]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (lane + 32 * u < nv) add_vec<DT, T>(col, v[u], emax);
      reg_left -= U * EPV;
      if (reg_left <= 0) {
        regularise<DT, T>(col);
        reg_left = REG_EVERY;
      }
    }
    if (!ok) {
      // copies for batches k .. min(k + S, nb) - 1 may still be in flight
      if (lane == 0) {
        for (int64_t j = k; j < nb && j < k + S; ++j) {
          const uint32_t gj = g + (uint32_t)j;
          mbar_wait(&full[gj % S], (gj / S) & 1u);
        }
        atomicOr(a.status, STATUS_TIMEOUT);
      }
      __syncwarp();
      return;
    }
    g += (uint32_t)nb;
    if (lane < r.tail_n) add_one<DT, T>(col, load_one<DT>(a.x, r.tail_lo + lane), emax);
    seg_finish_tile<DT, T, W>(a, w, r, digits, col, wacc, wlimbs, emax);
  }
}

// Windowed reducer: the windowed tile reduction of window.cuh in a
// persistent loop over the tile queue.
template <int DT, int W, int U>
__global__ void __launch_bounds__(W * 32, 1) seg_sum_kernel_win(SegArgs a) {
  constexpr int T = W * 32;
  constexpr int NC = win_rows<DT>();
  constexpr int ND = win_over_digits<DT>();
  extern __shared__ int64_t smem_win[];
  int64_t* cols = smem_win;                    // NC x T
  int64_t* overflow = smem_win + NC * T;       // W x ND
  __shared__ int64_t wacc[W][ACC_WORDS];
  __shared__ uint32_t wlimbs[W][ACC_DIGITS];

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int64_t* col = cols + t;
  int64_t* ov = overflow + warp * ND;
  for (int i = 0; i < NC; ++i) col[i * T] = 0;
  for (int i = lane; i < ND; i += 32) ov[i] = 0;
  __syncwarp();
  const int64_t total = (int64_t)__ldcg((const unsigned long long*)&a.counters[CNT_TOTAL]);
  if (total > a.map_capacity) return;  // flagged by the planner; results are NaN

  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(&a.counters[CNT_QUEUE], 1ull);
    const int64_t tile = (int64_t)__shfl_sync(0xffffffffu, tk, 0);
    if (tile >= total) break;
    const TileWork w = tile_work(a, tile);
    int64_t d0, d1, d2;
    uint32_t flags;
    win_tile<DT, T, U>(a.x, w.lo, w.hi, cols, ov, d0, d1, d2, flags);
    if (lane + 64 >= ACC_DIGITS) d2 = (lane + 64 < ACC_WORDS) ? flag_word(lane + 64, flags, w.hi - w.lo) : 0;
    seg_emit<DT, W, true>(a, w, d0, d1, d2, wacc, wlimbs);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int DT, int W>
static cudaError_t set_attr_t() {
  constexpr int U = 4;
  constexpr size_t SMEM = (size_t)Geometry<DT>::DIGITS * W * 32 * sizeof(int64_t);
  return cudaFuncSetAttribute(seg_sum_kernel<DT, W, U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SMEM);
}

// TMA reducer shapes: 2 stages of 8 vectors per lane; 8 warps for FP64
// (66-digit columns), 12 for FP32/BF16 (33-digit columns).
#ifndef ES_SEGTMA_F64_U
#define ES_SEGTMA_F64_U 10
#endif
#ifndef ES_SEGTMA_F64_S
#define ES_SEGTMA_F64_S 2
#endif
template <int DT> struct SegTma;
template <> struct SegTma<F64> { static constexpr int W = 8, U = ES_SEGTMA_F64_U, S = ES_SEGTMA_F64_S; };
template <> struct SegTma<F32> { static constexpr int W = 12, U = 8, S = 2; };
template <> struct SegTma<BF16> { static constexpr int W = 12, U = 8, S = 2; };

template <int DT>
constexpr size_t seg_tma_smem() {
  using C = SegTma<DT>;
  return (size_t)Geometry<DT>::DIGITS * C::W * 32 * 8 + (size_t)C::W * C::S * 32 * C::U * 16 +
         (size_t)C::W * C::S * 8;
}

template <int DT>
static cudaError_t set_attr_tma_t() {
  using C = SegTma<DT>;
  static_assert(seg_tma_smem<DT>() + (size_t)C::W * (ACC_WORDS * 8 + ACC_DIGITS * 4) <= 232448,
                "shared memory per CTA");
  return cudaFuncSetAttribute(seg_sum_kernel_tma<DT, C::W, C::U, C::S>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)seg_tma_smem<DT>());
}

template <int DT, int W>
static void launch_main_direct(const SegArgs& a, int grid, cudaStream_t st) {
  constexpr int U = 4;
  constexpr size_t SMEM = (size_t)Geometry<DT>::DIGITS * W * 32 * sizeof(int64_t);
  seg_sum_kernel<DT, W, U><<<grid, W * 32, SMEM, st>>>(a);
}

template <int DT>
constexpr size_t seg_win_smem() {
  using C = WinGeom<DT>;
  return (size_t)(C::WD + 1) * C::W * 32 * 8 + (size_t)C::W * Geometry<DT>::DIGITS * 8;
}

template <int DT>
static cudaError_t set_attr_win_t() {
  using C = WinGeom<DT>;
  static_assert(seg_win_smem<DT>() + (size_t)C::W * (ACC_WORDS * 8 + ACC_DIGITS * 4) <= 232448,
                "shared memory per CTA");
  return cudaFuncSetAttribute(seg_sum_kernel_win<DT, C::W, C::U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)seg_win_smem<DT>());
}

template <int DT>
static void launch_main_win(const SegArgs& a, int grid, cudaStream_t st) {
  using C = WinGeom<DT>;
  seg_sum_kernel_win<DT, C::W, C::U><<<grid, C::W * 32, seg_win_smem<DT>(), st>>>(a);
}

template <int DT>
static void launch_main_tma(const SegArgs& a, int grid, cudaStream_t st) {
  using C = SegTma<DT>;
  seg_sum_kernel_tma<DT, C::W, C::U, C::S><<<grid, C::W * 32, seg_tma_smem<DT>(), st>>>(a);
}

static cudaError_t configure_kernels(int dev) {
  // Several host threads may reach this at once (the handle-free entry point
  // has no handle to lock): the attribute calls are idempotent, and the flag
  // is atomic, so concurrent first calls at worst configure twice.
  static std::atomic<bool> done[64] = {};
  if (dev >= 0 && dev < 64 && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  cudaError_t e;
  if ((e = set_attr_t<F64, 8>()) != cudaSuccess) return e;
  if ((e = set_attr_t<F64, 12>()) != cudaSuccess) return e;
  if ((e = set_attr_t<F32, 8>()) != cudaSuccess) return e;
  if ((e = set_attr_t<F32, 16>()) != cudaSuccess) return e;
  if ((e = set_attr_t<BF16, 8>()) != cudaSuccess) return e;
  if ((e = set_attr_t<BF16, 16>()) != cudaSuccess) return e;
  if ((e = set_attr_tma_t<F64>()) != cudaSuccess) return e;
  if ((e = set_attr_tma_t<F32>()) != cudaSuccess) return e;
  if ((e = set_attr_tma_t<BF16>()) != cudaSuccess) return e;
  if ((e = set_attr_win_t<F64>()) != cudaSuccess) return e;
  if ((e = set_attr_win_t<F32>()) != cudaSuccess) return e;
  if ((e = set_attr_win_t<BF16>()) != cudaSuccess) return e;
  if (dev >= 0 && dev < 64) done[dev].store(true, std::memory_order_release);
  return cudaSuccess;
}

cudaError_t seg_preload() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = configure_kernels(dev);
  cudaFuncAttributes at;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&at, (const void*)seg_count_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&at, (const void*)seg_scan_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&at, (const void*)seg_base_kernel);
  return e;
}

int seg_warps_choice(int in_dt, int idx) {
  if (idx == 2) return in_dt == F64 ? SegTma<F64>::W : SegTma<F32>::W;
  if (idx == 3) return in_dt == F64 ? WinGeom<F64>::W : WinGeom<F32>::W;
  if (in_dt == F64) return idx == 0 ? 8 : 12;
  return idx == 0 ? 8 : 16;
}

cudaError_t seg_enqueue(int in_dt, const SegArgs& a, int warps, int kind, int num_sms, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = configure_kernels(dev)) != cudaSuccess) return e;
  const int64_t nblocks = (a.S + PLAN_T - 1) / PLAN_T;
  seg_count_kernel<<<(unsigned)nblocks, PLAN_T, 0, st>>>(a);
  seg_scan_kernel<<<1, PLAN_T, 0, st>>>(a, nblocks);
  seg_base_kernel<<<(unsigned)nblocks, PLAN_T, 0, st>>>(a);
  const int grid = num_sms;
  if (kind == SEG_KIND_WINDOW) {
    switch (in_dt) {
      case F64: launch_main_win<F64>(a, grid, st); break;
      case F32: launch_main_win<F32>(a, grid, st); break;
      default: launch_main_win<BF16>(a, grid, st); break;
    }
    return cudaGetLastError();
  }
  if (kind == SEG_KIND_TMA) {
    switch (in_dt) {
      case F64: launch_main_tma<F64>(a, grid, st); break;
      case F32: launch_main_tma<F32>(a, grid, st); break;
      default: launch_main_tma<BF16>(a, grid, st); break;
    }
    return cudaGetLastError();
  }
  switch (in_dt) {
    case F64:
      if (warps == 12) launch_main_direct<F64, 12>(a, grid, st);
      else launch_main_direct<F64, 8>(a, grid, st);
      break;
    case F32:
      if (warps == 16) launch_main_direct<F32, 16>(a, grid, st);
      else launch_main_direct<F32, 8>(a, grid, st);
      break;
    default:
      if (warps == 16) launch_main_direct<BF16, 16>(a, grid, st);
      else launch_main_direct<BF16, 8>(a, grid, st);
      break;
  }
  return cudaGetLastError();
}

}  // namespace es
