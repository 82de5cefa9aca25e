// stream.cuh -- the streaming inner loop shared by the single-array, the
// segmented and the serving kernels: read a thread's share of 16-byte
// vectors once (Section 5, Theorem 5: one scan, any order) and add their
// elements into the thread's private digit column.
#pragma once
#include <cstdint>

#include "digits.cuh"

namespace es {

__device__ __forceinline__ uint4 ldg_stream(const uint4* p) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p));
  return r;
}

// Ask the TMA unit to bring [p, p + bytes) into L2 ahead of the register
// loads (a hint: no data returns to the SM, no registers are held).  p and
// bytes must be multiples of 16.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

#ifndef ES_PREFETCH_BATCHES
#define ES_PREFETCH_BATCHES 0
#endif

__device__ __forceinline__ int64_t warp_sum(int64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Add vectors p[j * STEP], j in [0, cnt), into the digit column `col`
// (digit stride SSTRIDE).  U vectors per batch, two batches in flight
// (double buffered in registers).  `reg_left` counts additions until the
// next regularisation (Lemma 1 with deferred carries).
//
// The group of STEP threads that share this loop covers STEP*U contiguous
// vectors per batch and ends at `group_end`; its leader (idx == 0, whose p
// is the group's first vector) also prefetches the group's batch
// ES_PREFETCH_BATCHES ahead into L2, clamped to [p, group_end), so that more
// bytes are in flight than the registers can hold.
template <int DT, int SSTRIDE, int STEP, int U, typename D>
__device__ __forceinline__ void stream_add(D* __restrict__ col, const uint4* __restrict__ p,
                                           int64_t cnt, uint32_t& emax, int& reg_left, int idx,
                                           const uint4* group_end) {
  constexpr int EPV = 16 / Geometry<DT>::ELEM_BYTES;
  constexpr int REG_EVERY = RegEvery<DT, D>::value;
  constexpr int64_t PER = (int64_t)STEP * U;
  constexpr int PD = ES_PREFETCH_BATCHES;
  const int64_t nb = cnt / U;
  const uint4* p_end = group_end;  // only read by the leader
  if (PD > 0 && idx == 0) {
    for (int k = 0; k < PD; ++k) {
      const uint4* q = p + k * PER;
      if (q >= p_end) break;
      const int64_t n = min((int64_t)PER, (int64_t)(p_end - q));
      prefetch_l2(q, (uint32_t)(n * 16));
    }
  }
  uint4 A[U], B[U];
  if (nb > 0) {
#pragma unroll
    for (int u = 0; u < U; ++u) A[u] = ldg_stream(p + u * STEP);
  }
  for (int64_t k = 0; k < nb; k += 2) {
    if (PD > 0 && idx == 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint4* q = p + (k + PD + h) * PER;
        if (q < p_end) prefetch_l2(q, (uint32_t)(min((int64_t)PER, (int64_t)(p_end - q)) * 16));
      }
    }
    if (k + 1 < nb) {
#pragma unroll
      for (int u = 0; u < U; ++u) B[u] = ldg_stream(p + (k + 1) * PER + u * STEP);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) add_vec<DT, SSTRIDE>(col, A[u], emax);
    reg_left -= U * EPV;
    if (reg_left <= 0) {
      regularise<DT, SSTRIDE>(col);
      reg_left = REG_EVERY;
    }
    if (k + 1 >= nb) break;
    if (k + 2 < nb) {
#pragma unroll
      for (int u = 0; u < U; ++u) A[u] = ldg_stream(p + (k + 2) * PER + u * STEP);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) add_vec<DT, SSTRIDE>(col, B[u], emax);
    reg_left -= U * EPV;
    if (reg_left <= 0) {
      regularise<DT, SSTRIDE>(col);
      reg_left = REG_EVERY;
    }
  }
  for (int64_t j = nb * U; j < cnt; ++j) add_vec<DT, SSTRIDE>(col, ldg_stream(p + j * STEP), emax);
  reg_left -= (int)((cnt - nb * U) * EPV);
  if (reg_left <= 0) {
    regularise<DT, SSTRIDE>(col);
    reg_left = REG_EVERY;
  }
}

// Elements [lo, hi) of x split into an unaligned head (scalar, one element
// per lane), 16-byte vectors and a ragged tail (scalar).  Lane `lane` of a
// group of LANES threads takes head/tail element `lane` and vectors
// lane, lane + LANES, ...
struct RangeSplit {
  int64_t head_n;   // scalar elements before the first 16-byte boundary
  int64_t vlo;      // first element of the vector part
  int64_t nvec;     // vectors
  int64_t tail_lo;  // first tail element
  int64_t tail_n;   // tail elements
};

template <int DT>
__device__ __forceinline__ RangeSplit split_range(const void* x, int64_t lo, int64_t hi) {
  constexpr int EB = Geometry<DT>::ELEM_BYTES;
  constexpr int EPV = 16 / EB;
  RangeSplit r;
  const uintptr_t addr = (uintptr_t)x + (uintptr_t)(lo * EB);
  int64_t head = (int64_t)(((16u - (unsigned)(addr & 15u)) & 15u) / EB);
  const int64_t len = hi - lo;
  if (head > len) head = len;
  r.head_n = head;
  r.vlo = lo + head;
  r.nvec = (hi - r.vlo) / EPV;
  r.tail_lo = r.vlo + r.nvec * EPV;
  r.tail_n = hi - r.tail_lo;
  return r;
}

// Exact classification (specials, signed zeros) of one lane's elements of a
// split range; used only when the lane's exponent maximum says it matters.
template <int DT, int LANES>
__device__ uint32_t rescan_split(const void* x, const RangeSplit& r, int lane) {
  constexpr int EB = Geometry<DT>::ELEM_BYTES;
  constexpr int EPV = 16 / EB;
  uint32_t f = 0;
  if (lane < r.head_n) f |= classify<DT>(load_one<DT>(x, r.vlo - r.head_n + lane));
  for (int64_t v = lane; v < r.nvec; v += LANES)
    for (int e = 0; e < EPV; ++e) f |= classify<DT>(load_one<DT>(x, r.vlo + v * EPV + e));
  if (lane < r.tail_n) f |= classify<DT>(load_one<DT>(x, r.tail_lo + lane));
  return f;
}

// Add one lane's share of a split range into its column.
template <int DT, int SSTRIDE, int LANES, int U>
__device__ __forceinline__ void add_split(int64_t* __restrict__ col, const void* x, const RangeSplit& r,
                                          int lane, uint32_t& emax, int& reg_left) {
  constexpr int EB = Geometry<DT>::ELEM_BYTES;
  if (lane < r.head_n) add_one<DT, SSTRIDE>(col, load_one<DT>(x, r.vlo - r.head_n + lane), emax);
  const uint4* vp = reinterpret_cast<const uint4*>((const char*)x + r.vlo * EB);
  const int64_t cnt = (r.nvec > lane) ? (r.nvec - lane + LANES - 1) / LANES : 0;
  stream_add<DT, SSTRIDE, LANES, U>(col, vp + lane, cnt, emax, reg_left, lane, vp + r.nvec);
  if (lane < r.tail_n) add_one<DT, SSTRIDE>(col, load_one<DT>(x, r.tail_lo + lane), emax);
}

// Merge the regularised columns of one warp into a radix-2^32 accumulator:
// lane L returns digits L, L + 32 and (for L + 64 < ACC_DIGITS) L + 64.
// Column reads are rotated by lane so that no two lanes hit one bank pair.
template <int DT, int SSTRIDE>
__device__ __forceinline__ void warp_merge(const int64_t* warp_cols, int lane, int64_t& d0, int64_t& d1,
                                           int64_t& d2) {
  d0 = d1 = d2 = 0;
#pragma unroll 4
  for (int k = 0; k < 32; ++k) {
    const int64_t* c = warp_cols + ((k + lane) & 31);
    d0 += digit32<DT, SSTRIDE>(c, lane);
    d1 += digit32<DT, SSTRIDE>(c, lane + 32);
    if (lane + 64 < ACC_DIGITS) d2 += digit32<DT, SSTRIDE>(c, lane + 64);
  }
}

// Word w (>= ACC_DIGITS) of an accumulator from flag bits and a count.
__device__ __forceinline__ int64_t flag_word(int w, uint32_t flags, int64_t count) {
  switch (w) {
    case W_NAN: return (flags & 1u) ? 1 : 0;
    case W_PINF: return (flags & 2u) ? 1 : 0;
    case W_NINF: return (flags & 4u) ? 1 : 0;
    case W_NOTPZ: return (flags & 8u) ? 1 : 0;
    case W_NOTNZ: return (flags & 16u) ? 1 : 0;
    case W_COUNT: return count;
    default: return 0;
  }
}

}  // namespace es
