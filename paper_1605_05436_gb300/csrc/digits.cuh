// digits.cuh -- per-element conversion into superaccumulator digits and the
// carry-free digit arithmetic of Section 2 (Lemma 1), for sm_103a.
//
// Representation.  Every input element is x = (-1)^s * m * 2^p * unit, where
// for a finite input with biased exponent E and stored fraction F:
//     m = F            if E == 0 (subnormal or zero), else F + 2^t,
//     p = max(E, 1) - 1,
// and unit is the format's smallest subnormal (2^-1074, 2^-149, 2^-133).
// The running sum is kept as a vector of signed 64-bit digits D_i with
// value sum_i D_i * 2^(r*i) * unit, where r is the digit radix in bits.  This
// is the integer-digit form of the (alpha, beta)-regularised superaccumulator
// (Section 2: y_i = Y_i R^i with integer Y_i, consecutive digits overlapping),
// with R = 2^r and a much wider overlap than one bit: a digit may hold many
// un-carried additions before it has to be regularised.
//
//   FP64:   r = 32.  m < 2^53 and p & 31 < 32, so m * 2^(p & 31) < 2^84
//           splits into a low part < 2^32 (digit p >> 5) and a high part
//           < 2^52 (digit (p >> 5) + 1): two digit additions per element.
//           66 digits per thread (digit 65 only receives carries).
//   FP32:   r = 8.   m < 2^24, so m * 2^(p & 7) < 2^31 goes into one digit
//   BF16:            (p >> 3) without splitting.  33 digits per thread.
//
// The single-array FP32 and BF16 kernels use sign-split unsigned columns
// instead (positive and negative elements in separate halves, so an element
// needs no sign arithmetic): FP32 radix 2^32 in overlapping 64-bit digits
// (radix 2^16 selectable), BF16 radix 2^8 in 32-bit digits, each defined
// below with its decode.
//
// Regularisation (Lemma 1, generalised to deferred carries): a digit D is
// replaced by D - c * R and its upper neighbour gains c, with
// c = floor((D + R/2) / R) (the balanced choice; Lemma 1 allows any signed
// carry that brings the digit into range).  Carries only ever move to the
// adjacent digit.
#pragma once
#include <cstdint>

namespace es {

enum : int { F64 = 0, F32 = 1, BF16 = 2 };
enum : int { RNE = 0, RTZ = 1, RUP = 2, RDOWN = 3 };

constexpr int ACC_DIGITS = 72;  // radix-2^32 digits of a merged accumulator
constexpr int ACC_WORDS = 80;   // digits + 5 counters + count + 2 reserved
constexpr int W_NAN = 72, W_PINF = 73, W_NINF = 74, W_NOTPZ = 75, W_NOTNZ = 76, W_COUNT = 77;

// Per-thread accumulator geometry by input format.
template <int DT> struct Geometry;
template <> struct Geometry<F64> {
  static constexpr int RADIX_BITS = 32;
  static constexpr int DIGITS = 66;           // per-thread digits
  static constexpr int ELEM_BYTES = 8;
#ifndef ES_F64_REG_EVERY
#define ES_F64_REG_EVERY 1984
#endif
  // adds between regularisations: after one, |digit| <= 2^31 + 2^21, and each
  // add changes a digit by at most 2^52, so up to 2047 adds stay below 2^63
  // (callers check after each batch of at most 16 adds, plus 2 scalar adds)
  static constexpr int REG_EVERY = ES_F64_REG_EVERY;
  static constexpr uint32_t EXP_SPECIAL = 0x7FF;
};
template <> struct Geometry<F32> {
  static constexpr int RADIX_BITS = 8;
  static constexpr int DIGITS = 33;
  static constexpr int ELEM_BYTES = 4;
  static constexpr int REG_EVERY = 1 << 30;   // |add| < 2^31: int64 holds 2^32 of them
  static constexpr uint32_t EXP_SPECIAL = 0xFF;
};
template <> struct Geometry<BF16> {
  static constexpr int RADIX_BITS = 8;
  static constexpr int DIGITS = 33;
  static constexpr int ELEM_BYTES = 2;
  static constexpr int REG_EVERY = 1 << 30;
  static constexpr uint32_t EXP_SPECIAL = 0xFF;
};

__host__ __device__ constexpr int unit_exp_of(int dt) {
  return dt == F64 ? -1074 : (dt == F32 ? -149 : -133);
}

// ---------------------------------------------------------------------------
// Per-element conversion and digit addition (Section 3 step 2 / Section 5
// step 1: split each element into O(1) components at radix-aligned
// exponents; Section 5 Theorem 5: add them into the resident accumulator in
// any order).  `col` points at this thread's digit 0; digit i lives at
// col[i * STRIDE] (digit-major, thread-minor: conflict-free shared banks).
// `emax` tracks the largest biased exponent seen, which flags specials
// (E all ones) and all-zero/subnormal inputs for a later exact rescan.
// ---------------------------------------------------------------------------
// d += v on a digit of a thread-private shared-memory column.  (A
// shared-memory reduction, red.shared.add.u64, measured 35% slower here than
// the plain load / add / store.)
__device__ __forceinline__ void digit_add(int64_t* d, int64_t v) { *d += v; }

#ifndef ES_DECODE_V2
#define ES_DECODE_V2 0
#endif
#ifndef ES_P_FUSED
#define ES_P_FUSED 0
#endif

// Element decode and digit addition with the biased exponent E already
// extracted.  The hidden bit (set iff E >= 1) is a select on E.  (The
// ES_DECODE_V2 form takes it from bit 11 (FP64) or bit 8 (FP32) of
// E + all-ones, moved into place by a multiply on the FMA pipe; it measured
// 12% slower.)
template <int STRIDE>
__device__ __forceinline__ void add_f64_e(int64_t* __restrict__ col, uint32_t lo, uint32_t hi, uint32_t E) {
#if ES_DECODE_V2
  const uint32_t t = E * 512u + (0x7FFu << 9);          // bit 20 = (E >= 1); bits > 20 clear
  const uint32_t mhi = (hi & 0xFFFFFu) | (t & ~0xFFFFFu);  // bits 32..52 of m
#else
  const uint32_t mhi = (hi & 0xFFFFFu) | (E != 0u ? 0x100000u : 0u);
#endif
#if ES_P_FUSED
  const uint32_t p = (uint32_t)max((int)E - 1, 0);
#else
  const uint32_t p = max(E, 1u) - 1u;
#endif
  // v = m << (p & 31) is built as three 32-bit words w2:w1:w0 by funnel
  // shifts (which use p & 31).  The sign is applied before the shifts: the
  // funnel shifts of (sm : mhi^sm : lo^sm), sm = 0 or all ones, give v for a
  // positive element and its 96-bit complement ~v = -v - 1 for a negative
  // one (the fill bits are sm).  The low digit then gains w0 plus the sign
  // bit (one three-input add), the high digit the signed 64-bit w2:w1:
  //   -v = (2^32 - 1 - (v mod 2^32) + 1) + (-(v >> 32) - 1) * 2^32.
  // Contributions: low digit in [0, 2^32], high digit in [-2^52, 2^52).
  // (Measured against negating after the shifts: 2% faster; against a
  // separate 96-bit negation: 6% faster.  Moving the high-digit add to the
  // FMA pipe as a 32 x 32 -> 64-bit multiply-add by 1 measured 11% slower.)
  const uint32_t sm = (uint32_t)((int32_t)hi >> 31);
  const uint32_t xl = lo ^ sm, xh = mhi ^ sm;
  const uint32_t w0 = __funnelshift_l(sm, xl, p);
  const uint32_t w1 = __funnelshift_l(xl, xh, p);
  const uint32_t w2 = __funnelshift_l(xh, sm, p);
  int64_t* d = col + (p >> 5) * STRIDE;
  digit_add(d, (int64_t)((uint64_t)w0 + (hi >> 31)));
  digit_add(d + STRIDE, (int64_t)(((uint64_t)w2 << 32) | w1));
}

template <int STRIDE>
__device__ __forceinline__ void add_f64(int64_t* __restrict__ col, uint32_t lo, uint32_t hi,
                                        uint32_t& emax) {
  const uint32_t E = (hi >> 20) & 0x7FFu;
  emax = max(emax, E);
  add_f64_e<STRIDE>(col, lo, hi, E);
}

template <int STRIDE>
__device__ __forceinline__ void add_f32_e(int64_t* __restrict__ col, uint32_t w, uint32_t E) {
#if ES_DECODE_V2
  const uint32_t t = E * 32768u + (0xFFu << 15);         // bit 23 = (E >= 1); bits > 23 clear
  const uint32_t m = (w & 0x7FFFFFu) | (t & ~0x7FFFFFu);
  const uint32_t p = (uint32_t)max((int)E - 1, 0);
#else
  const uint32_t m = (w & 0x7FFFFFu) | (E != 0u ? 0x800000u : 0u);
  const uint32_t p = max(E, 1u) - 1u;
#endif
  const int32_t s = (int32_t)w >> 31;
  const int32_t v = ((int32_t)(m << (p & 7u)) ^ s) - s;  // |v| < 2^31
  digit_add(col + (p >> 3) * STRIDE, (int64_t)v);
}

template <int STRIDE>
__device__ __forceinline__ void add_f32(int64_t* __restrict__ col, uint32_t w, uint32_t& emax) {
  const uint32_t E = (w >> 23) & 0xFFu;
  emax = max(emax, E);
  add_f32_e<STRIDE>(col, w, E);
}

template <int STRIDE>
__device__ __forceinline__ void add_bf16_e(int64_t* __restrict__ col, uint32_t h, uint32_t E) {
#if ES_DECODE_V2
  const uint32_t m = (h & 0x7Fu) | (min(E, 1u) * 128u);
  const uint32_t p = (uint32_t)max((int)E - 1, 0);
#else
  const uint32_t m = (h & 0x7Fu) | (E != 0u ? 0x80u : 0u);
  const uint32_t p = max(E, 1u) - 1u;
#endif
  const int32_t s = -(int32_t)((h >> 15) & 1u);
  const int32_t v = ((int32_t)(m << (p & 7u)) ^ s) - s;  // |v| < 2^15
  digit_add(col + (p >> 3) * STRIDE, (int64_t)v);
}

template <int STRIDE>
__device__ __forceinline__ void add_bf16(int64_t* __restrict__ col, uint32_t h, uint32_t& emax) {
  const uint32_t E = (h >> 7) & 0xFFu;
  emax = max(emax, E);
  add_bf16_e<STRIDE>(col, h, E);
}

// Add all elements held in one 16-byte vector.  The exponent maximum is
// updated with three-input maxima, once per vector.
template <int DT, int STRIDE>
__device__ __forceinline__ void add_vec(int64_t* __restrict__ col, const uint4& v, uint32_t& emax) {
  if constexpr (DT == F64) {
    const uint32_t e0 = (v.y >> 20) & 0x7FFu, e1 = (v.w >> 20) & 0x7FFu;
    emax = __vimax3_u32(emax, e0, e1);
    add_f64_e<STRIDE>(col, v.x, v.y, e0);
    add_f64_e<STRIDE>(col, v.z, v.w, e1);
  } else if constexpr (DT == F32) {
    const uint32_t e0 = (v.x >> 23) & 0xFFu, e1 = (v.y >> 23) & 0xFFu;
    const uint32_t e2 = (v.z >> 23) & 0xFFu, e3 = (v.w >> 23) & 0xFFu;
    emax = __vimax3_u32(__vimax3_u32(emax, e0, e1), e2, e3);
    add_f32_e<STRIDE>(col, v.x, e0);
    add_f32_e<STRIDE>(col, v.y, e1);
    add_f32_e<STRIDE>(col, v.z, e2);
    add_f32_e<STRIDE>(col, v.w, e3);
  } else {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t e[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      e[2 * k] = (w[k] >> 7) & 0xFFu;
      e[2 * k + 1] = (w[k] >> 23) & 0xFFu;
    }
    emax = __vimax3_u32(__vimax3_u32(emax, e[0], e[1]), __vimax3_u32(e[2], e[3], e[4]),
                        __vimax3_u32(e[5], e[6], e[7]));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      add_bf16_e<STRIDE>(col, w[k] & 0xFFFFu, e[2 * k]);
      add_bf16_e<STRIDE>(col, w[k] >> 16, e[2 * k + 1]);
    }
  }
}

// Add one element given by its raw bits (for unaligned heads and tails).
template <int DT, int STRIDE>
__device__ __forceinline__ void add_one(int64_t* __restrict__ col, uint64_t bits, uint32_t& emax) {
  if constexpr (DT == F64) add_f64<STRIDE>(col, (uint32_t)bits, (uint32_t)(bits >> 32), emax);
  else if constexpr (DT == F32) add_f32<STRIDE>(col, (uint32_t)bits, emax);
  else add_bf16<STRIDE>(col, (uint32_t)bits, emax);
}

template <int DT>
__device__ __forceinline__ uint64_t load_one(const void* x, int64_t i) {
  if constexpr (DT == F64) return __ldg((const unsigned long long*)x + i);
  else if constexpr (DT == F32) return __ldg((const unsigned int*)x + i);
  else return __ldg((const unsigned short*)x + i);
}

// Regularise one thread's digits in place: afterwards |D_i| <= R/2 for all
// but the top digit, which absorbs the last carry.
template <int DT, int STRIDE>
__device__ __forceinline__ void regularise(int64_t* __restrict__ col) {
  constexpr int RB = Geometry<DT>::RADIX_BITS;
  constexpr int ND = Geometry<DT>::DIGITS;
  int64_t carry = 0;
#pragma unroll 4
  for (int i = 0; i < ND - 1; ++i) {
    const int64_t v = col[i * STRIDE] + carry;
    const int64_t c = (v + ((int64_t)1 << (RB - 1))) >> RB;
    col[i * STRIDE] = v - (c << RB);
    carry = c;
  }
  col[(ND - 1) * STRIDE] += carry;
}

// Value of radix-2^32 digit i contributed by one thread's (regularised)
// digits: for FP64 it is digit i itself; for the radix-2^8 formats it
// gathers digits 4i .. 4i+3.
template <int DT, int STRIDE>
__device__ __forceinline__ int64_t digit32(const int64_t* __restrict__ col, int i) {
  constexpr int ND = Geometry<DT>::DIGITS;
  if constexpr (DT == F64) {
    return i < ND ? col[i * STRIDE] : 0;
  } else {
    int64_t v = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int j = 4 * i + k;
      if (j < ND) v += col[j * STRIDE] * ((int64_t)1 << (8 * k));
    }
    return v;
  }
}

// ---------------------------------------------------------------------------
// BF16 with 32-bit digits.  A BF16 element adds less than 2^15 to one
// radix-2^8 digit, so an int32 digit regularised to |D| <= 2^7 takes 65,000
// more additions before it could overflow: half the shared-memory traffic
// and a quarter of the column footprint of the int64 form.
// ---------------------------------------------------------------------------
template <int STRIDE>
__device__ __forceinline__ void add_bf16_e(int32_t* __restrict__ col, uint32_t h, uint32_t E) {
  const uint32_t m = (h & 0x7Fu) | (E != 0u ? 0x80u : 0u);
  const uint32_t p = max(E, 1u) - 1u;
  // the signed addition as a multiply-add by +-1 (FMA pipe), which frees
  // the integer ALU pipe that bounds this kernel (measured 6% faster; the
  // 64-bit form, mad.wide.s32, measured 3% slower for FP32)
  // (a byte-permute with sign replication for the sign measured 3% slower)
  const int32_t sgn = ((int32_t)(h << 16) >> 31) | 1;
  int32_t* d = col + (p >> 3) * STRIDE;
  int32_t a = *d;
  asm("mad.lo.s32 %0, %1, %2, %0;" : "+r"(a) : "r"((int32_t)(m << (p & 7u))), "r"(sgn));
  *d = a;
}

template <int DT, int STRIDE>
__device__ __forceinline__ void add_vec(int32_t* __restrict__ col, const uint4& v, uint32_t& emax) {
  static_assert(DT == BF16, "32-bit digit columns hold BF16 sums only");
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint32_t e[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    e[2 * k] = (w[k] >> 7) & 0xFFu;
    e[2 * k + 1] = (w[k] >> 23) & 0xFFu;
  }
  emax = __vimax3_u32(__vimax3_u32(emax, e[0], e[1]), __vimax3_u32(e[2], e[3], e[4]),
                      __vimax3_u32(e[5], e[6], e[7]));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    add_bf16_e<STRIDE>(col, w[k] & 0xFFFFu, e[2 * k]);
    add_bf16_e<STRIDE>(col, w[k] >> 16, e[2 * k + 1]);
  }
}

template <int DT, int STRIDE>
__device__ __forceinline__ void add_one(int32_t* __restrict__ col, uint64_t bits, uint32_t& emax) {
  static_assert(DT == BF16, "32-bit digit columns hold BF16 sums only");
  const uint32_t h = (uint32_t)bits & 0xFFFFu;
  const uint32_t E = (h >> 7) & 0xFFu;
  emax = max(emax, E);
  add_bf16_e<STRIDE>(col, h, E);
}

template <int DT, int STRIDE>
__device__ __forceinline__ void regularise(int32_t* __restrict__ col) {
  static_assert(DT == BF16, "32-bit digit columns hold BF16 sums only");
  constexpr int ND = Geometry<DT>::DIGITS;
  int32_t carry = 0;
#pragma unroll 4
  for (int i = 0; i < ND - 1; ++i) {
    const int32_t v = col[i * STRIDE] + carry;
    const int32_t c = (v + 128) >> 8;
    col[i * STRIDE] = v - (c << 8);
    carry = c;
  }
  col[(ND - 1) * STRIDE] += carry;
}

template <int DT, int STRIDE>
__device__ __forceinline__ int64_t digit32(const int32_t* __restrict__ col, int i) {
  static_assert(DT == BF16, "32-bit digit columns hold BF16 sums only");
  constexpr int ND = Geometry<DT>::DIGITS;
  int64_t v = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = 4 * i + k;
    if (j < ND) v += (int64_t)col[j * STRIDE] * ((int64_t)1 << (8 * k));
  }
  return v;
}

// ---------------------------------------------------------------------------
// BF16 with sign-split columns: a thread's column holds two halves of
// unsigned 32-bit digits, positive elements adding into digits 0..32 and
// negative ones into digits 33..65, so that an element costs no sign
// arithmetic at all: its sign bit only selects the half (an integer
// multiply-add in the address, on the FMA pipe).  The column's value is the
// positive half minus the negative half.  Regularisation carries upwards
// within each half (digits end in [0, 255]); the top digit of a half
// receives at most 2^7 per element of the thread's share, below 2^32 for any
// array that fits in memory.  (Measured 2% faster than signed int32 digits
// with a multiply-add by +-1; the same split for FP32, whose 64-bit digits
// then need 528 B per thread, measured 17% slower for want of threads.)
// ---------------------------------------------------------------------------
template <int DT, typename D>
struct ColumnDigits {
  static constexpr int value = Geometry<DT>::DIGITS;
};
template <int DT>
struct ColumnDigits<DT, uint32_t> {
  static constexpr int value = 2 * Geometry<DT>::DIGITS;
};

// h < 2^16: its bit 15 is the sign
template <int STRIDE>
__device__ __forceinline__ void add_bf16_split(uint32_t* __restrict__ col, uint32_t h, uint32_t E) {
  const uint32_t m = (h & 0x7Fu) | (E != 0u ? 0x80u : 0u);
  const uint32_t p = max(E, 1u) - 1u;
  col[((p >> 3) + (h >> 15) * 33u) * STRIDE] += m << (p & 7u);
}

#ifndef ES_BF16_PACKED
#define ES_BF16_PACKED 1
#endif

template <int DT, int STRIDE>
__device__ __forceinline__ void add_vec(uint32_t* __restrict__ col, const uint4& v, uint32_t& emax) {
  static_assert(DT == BF16, "sign-split 32-bit columns hold BF16 sums only");
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#if ES_BF16_PACKED
  // Both elements of a 32-bit word decoded at once in 16-bit halves (the
  // exponent in bits 0-7 and 16-23): p = max(E - 1, 0) by one add-max of
  // 16-bit pairs, the sign half offset (33 digits = 264 bit positions)
  // folded into p, the digit index and the in-digit shift extracted per half.
  // (Measured 17% faster than decoding each element on its own; keeping the
  // exponent maximum packed, 2% more; the direct upper index and the masked
  // funnel-shift amounts, 5% more.)
  uint32_t E2[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) E2[k] = (w[k] >> 7) & 0x00FF00FFu;
  // the running maximum stays packed in 16-bit halves (emax_unpack)
  emax = __vimax3_u16x2(__vimax3_u16x2(emax, E2[0], E2[1]), E2[2], E2[3]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t p2 = __viaddmax_s16x2(E2[k], 0xFFFFFFFFu, 0u);          // max(E - 1, 0)
    const uint32_t q2 = p2 + ((w[k] >> 15) & 0x00010001u) * 264u;         // + 33 digits if negative
    const uint32_t m2 = (w[k] & 0x007F007Fu) | (__vimin3_u16x2(E2[k], 0x00010001u, 0x00010001u) << 7);
    // digit indices: q < 2^10 in each half, so the upper one is q2 >> 19;
    // both in-digit shifts from one masked word, applied by wrap-mode funnel
    // shifts (which use the amount mod 32: bits 3-4 are clear)
    const uint32_t i0 = (q2 >> 3) & 0xFFu, i1 = q2 >> 19;
    const uint32_t s2 = q2 & 0x00070007u;
    col[i0 * STRIDE] += __funnelshift_l(0u, m2 & 0xFFu, s2);
    col[i1 * STRIDE] += __funnelshift_l(0u, m2 >> 16, s2 >> 16);
  }
#else
  uint32_t e[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    e[2 * k] = (w[k] >> 7) & 0xFFu;
    e[2 * k + 1] = (w[k] >> 23) & 0xFFu;
  }
  emax = __vimax3_u32(__vimax3_u32(emax, e[0], e[1]), __vimax3_u32(e[2], e[3], e[4]),
                      __vimax3_u32(e[5], e[6], e[7]));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    add_bf16_split<STRIDE>(col, w[k] & 0xFFFFu, e[2 * k]);
    add_bf16_split<STRIDE>(col, w[k] >> 16, e[2 * k + 1]);
  }
#endif
}

template <int DT, int STRIDE>
__device__ __forceinline__ void add_one(uint32_t* __restrict__ col, uint64_t bits, uint32_t& emax) {
  static_assert(DT == BF16, "sign-split 32-bit columns hold BF16 sums only");
  const uint32_t h = (uint32_t)bits & 0xFFFFu;
  const uint32_t E = (h >> 7) & 0xFFu;
  emax = max(emax, E);
  add_bf16_split<STRIDE>(col, h, E);
}

template <int DT, int STRIDE>
__device__ __forceinline__ void regularise(uint32_t* __restrict__ col) {
  static_assert(DT == BF16, "sign-split 32-bit columns hold BF16 sums only");
  constexpr int ND = Geometry<DT>::DIGITS;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t* c = col + h * ND * STRIDE;
    uint32_t carry = 0;
#pragma unroll 4
    for (int i = 0; i < ND - 1; ++i) {
      const uint32_t v = c[i * STRIDE] + carry;
      c[i * STRIDE] = v & 0xFFu;
      carry = v >> 8;
    }
    c[(ND - 1) * STRIDE] += carry;
  }
}
template <int DT, int STRIDE>
__device__ __forceinline__ int64_t digit32(const uint32_t* __restrict__ col, int i) {
  static_assert(DT == BF16, "sign-split 32-bit columns hold BF16 sums only");
  constexpr int ND = Geometry<DT>::DIGITS;
  int64_t v = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = 4 * i + k;
    if (j < ND) v += ((int64_t)col[j * STRIDE] - (int64_t)col[(ND + j) * STRIDE]) * ((int64_t)1 << (8 * k));
  }
  return v;
}

#ifndef ES_F32_R32
#define ES_F32_R32 1
#endif
#if ES_F32_R32
// ---------------------------------------------------------------------------
// FP32 with radix-2^32 sign-split columns (uint64_t digits): an element adds
// m << (p & 31) (< 2^55, whole, no split) into digit (p >> 5) of its half
// (positive and negative elements in separate halves, so no sign
// arithmetic).  Digits overlap: each holds up to 64 bits, and a
// regularisation (every F32_R32_REG_EVERY additions) moves everything above
// bit 32 into the next digit.  8 digits take elements (p >> 5 <= 7), two
// more take carries (the sum of n elements is below 2^(277 + log2 n)), so
// the two halves take 160 B per thread.  The shift amount is the packed
// exponent word as it is: a funnel shift uses its low five bits, p & 31.
// ---------------------------------------------------------------------------
constexpr int F32_R32_DIGITS = 10;
// after a regularisation every digit is below 2^32; with at most 511 more
// additions of less than 2^55 it stays below 2^64 (the callers check after
// each batch of at most 64 additions, plus a few scalar ones)
constexpr int F32_R32_REG_EVERY = 400;
template <>
struct ColumnDigits<F32, uint64_t> {
  static constexpr int value = 2 * F32_R32_DIGITS;
};

template <int STRIDE>
__device__ __forceinline__ void add_f32_r32(uint64_t* __restrict__ col, uint32_t w, uint32_t E) {
  const uint32_t m = (w & 0x7FFFFFu) | (E != 0u ? 0x800000u : 0u);
  const uint32_t p = max(E, 1u) - 1u;
  col[((p >> 5) + (w >> 31) * (uint32_t)F32_R32_DIGITS) * STRIDE] += (uint64_t)m << (p & 31u);
}

// Two FP32 elements decoded together in 16-bit halves, as in the radix-2^16
// form below; m << (p & 31) as two funnel shifts of m by the packed word
// (the lower element's shift: its low five bits; the upper one's: the word
// shifted down by 16).
template <int STRIDE>
__device__ __forceinline__ void add_f32_r32_pair(uint64_t* __restrict__ col, uint32_t w0, uint32_t w1,
                                                 uint32_t& emax2) {
  const uint32_t hh = __byte_perm(w0, w1, 0x7632);      // (w0 >> 16) | (w1 & 0xFFFF0000)
  const uint32_t E2 = (hh >> 7) & 0x00FF00FFu;          // E of w0 in bits 0-7, of w1 in bits 16-23
  emax2 = __vimax3_u16x2(emax2, E2, E2);
  const uint32_t p2 = __viaddmax_s16x2(E2, 0xFFFFFFFFu, 0u);       // max(E - 1, 0) per half
  const uint32_t hb2 = __vimin3_u16x2(E2, 0x00010001u, 0x00010001u);  // E >= 1 per half
  // digit p >> 5 of the element's half (negative elements: + F32_R32_DIGITS)
  const uint32_t q2 = ((p2 >> 5) & 0x00070007u) + ((hh >> 15) & 0x00010001u) * (uint32_t)F32_R32_DIGITS;
  const uint32_t m0 = (w0 & 0x7FFFFFu) | (hb2 << 23);
  const uint32_t m1 = (w1 & 0x7FFFFFu) | ((hb2 << 7) & 0x800000u);
  const uint32_t p1 = p2 >> 16;
  const uint64_t v0 = ((uint64_t)__funnelshift_l(m0, 0u, p2) << 32) | __funnelshift_l(0u, m0, p2);
  const uint64_t v1 = ((uint64_t)__funnelshift_l(m1, 0u, p1) << 32) | __funnelshift_l(0u, m1, p1);
  col[(q2 & 0xFFFFu) * STRIDE] += v0;
  col[(q2 >> 16) * STRIDE] += v1;
}

template <int DT, int STRIDE>
__device__ __forceinline__ void add_vec(uint64_t* __restrict__ col, const uint4& v, uint32_t& emax) {
  static_assert(DT == F32, "radix-2^32 split columns hold FP32 sums only");
  add_f32_r32_pair<STRIDE>(col, v.x, v.y, emax);
  add_f32_r32_pair<STRIDE>(col, v.z, v.w, emax);
}

template <int DT, int STRIDE>
__device__ __forceinline__ void add_one(uint64_t* __restrict__ col, uint64_t bits, uint32_t& emax) {
  static_assert(DT == F32, "radix-2^32 split columns hold FP32 sums only");
  const uint32_t w = (uint32_t)bits;
  const uint32_t E = (w >> 23) & 0xFFu;
  emax = max(emax, E);
  add_f32_r32<STRIDE>(col, w, E);
}

template <int DT, int STRIDE>
__device__ __forceinline__ void regularise(uint64_t* __restrict__ col) {
  static_assert(DT == F32, "radix-2^32 split columns hold FP32 sums only");
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint64_t* c = col + h * F32_R32_DIGITS * STRIDE;
    uint64_t carry = 0;
#pragma unroll 3
    for (int i = 0; i < F32_R32_DIGITS - 1; ++i) {
      const uint64_t v = c[i * STRIDE];
      const uint64_t lo = (v & 0xFFFFFFFFu) + carry;  // below 2^33
      c[i * STRIDE] = lo & 0xFFFFFFFFu;
      carry = (v >> 32) + (lo >> 32);
    }
    c[(F32_R32_DIGITS - 1) * STRIDE] += carry;
  }
}

// radix-2^32 digit i: positive half minus negative half
template <int DT, int STRIDE>
__device__ __forceinline__ int64_t digit32(const uint64_t* __restrict__ col, int i) {
  static_assert(DT == F32, "radix-2^32 split columns hold FP32 sums only");
  if (i >= F32_R32_DIGITS) return 0;
  return (int64_t)col[i * STRIDE] - (int64_t)col[(F32_R32_DIGITS + i) * STRIDE];
}
#else
// ---------------------------------------------------------------------------
// FP32 with radix-2^16 sign-split columns (uint64_t digits): 18 digits per
// half cover the 277-bit range, so the two halves (positive and negative
// elements) take 288 B per thread; an element adds m << (p & 15) (< 2^39,
// a 64-bit shift) into digit (p >> 4) of its half, with no sign arithmetic.
// ---------------------------------------------------------------------------
constexpr int F32_R16_DIGITS = 18;
template <>
struct ColumnDigits<F32, uint64_t> {
  static constexpr int value = 2 * F32_R16_DIGITS;
};

template <int STRIDE>
__device__ __forceinline__ void add_f32_r16(uint64_t* __restrict__ col, uint32_t w, uint32_t E) {
  const uint32_t m = (w & 0x7FFFFFu) | (E != 0u ? 0x800000u : 0u);
  const uint32_t p = max(E, 1u) - 1u;
  col[((p >> 4) + (w >> 31) * (uint32_t)F32_R16_DIGITS) * STRIDE] += (uint64_t)m << (p & 15u);
}

// Two FP32 elements decoded together in 16-bit halves: one byte permute
// brings both exponents (and both signs) into one word, then p = max(E - 1, 0)
// is one add-max of 16-bit pairs, the hidden bits one 16-bit-pair minimum,
// the digit index (half offset included) one add of pairs.  The running
// exponent maximum is kept as two 16-bit maxima packed in one word
// (emax_unpack gives the plain maximum).  (Measured 3.6% faster than
// decoding each element on its own; the same pairing measured 4% slower for
// FP64, whose 11-bit exponents and two-digit additions leave less to share.)
template <int STRIDE>
__device__ __forceinline__ void add_f32_r16_pair(uint64_t* __restrict__ col, uint32_t w0, uint32_t w1,
                                                 uint32_t& emax2) {
  const uint32_t hh = __byte_perm(w0, w1, 0x7632);      // (w0 >> 16) | (w1 & 0xFFFF0000)
  const uint32_t E2 = (hh >> 7) & 0x00FF00FFu;          // E of w0 in bits 0-7, of w1 in bits 16-23
  emax2 = __vimax3_u16x2(emax2, E2, E2);
  const uint32_t p2 = __viaddmax_s16x2(E2, 0xFFFFFFFFu, 0u);       // max(E - 1, 0) per half
  const uint32_t hb2 = __vimin3_u16x2(E2, 0x00010001u, 0x00010001u);  // E >= 1 per half
  // digit p >> 4 of the element's half (negative elements: + F32_R16_DIGITS)
  const uint32_t q2 = ((p2 >> 4) & 0x000F000Fu) + ((hh >> 15) & 0x00010001u) * (uint32_t)F32_R16_DIGITS;
  const uint32_t m0 = (w0 & 0x7FFFFFu) | (hb2 << 23);
  const uint32_t m1 = (w1 & 0x7FFFFFu) | ((hb2 << 7) & 0x800000u);
  col[(q2 & 0xFFFFu) * STRIDE] += (uint64_t)m0 << (p2 & 15u);
  col[(q2 >> 16) * STRIDE] += (uint64_t)m1 << ((p2 >> 16) & 15u);
}

template <int DT, int STRIDE>
__device__ __forceinline__ void add_vec(uint64_t* __restrict__ col, const uint4& v, uint32_t& emax) {
  static_assert(DT == F32, "radix-2^16 split columns hold FP32 sums only");
  add_f32_r16_pair<STRIDE>(col, v.x, v.y, emax);
  add_f32_r16_pair<STRIDE>(col, v.z, v.w, emax);
}

template <int DT, int STRIDE>
__device__ __forceinline__ void add_one(uint64_t* __restrict__ col, uint64_t bits, uint32_t& emax) {
  static_assert(DT == F32, "radix-2^16 split columns hold FP32 sums only");
  const uint32_t w = (uint32_t)bits;
  const uint32_t E = (w >> 23) & 0xFFu;
  emax = max(emax, E);
  add_f32_r16<STRIDE>(col, w, E);
}

template <int DT, int STRIDE>
__device__ __forceinline__ void regularise(uint64_t* __restrict__ col) {
  static_assert(DT == F32, "radix-2^16 split columns hold FP32 sums only");
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint64_t* c = col + h * F32_R16_DIGITS * STRIDE;
    uint64_t carry = 0;
#pragma unroll 3
    for (int i = 0; i < F32_R16_DIGITS - 1; ++i) {
      const uint64_t v = c[i * STRIDE] + carry;
      c[i * STRIDE] = v & 0xFFFFu;
      carry = v >> 16;
    }
    c[(F32_R16_DIGITS - 1) * STRIDE] += carry;
  }
}

// radix-2^32 digit i = radix-2^16 digits 2i and 2i + 1, positive half minus
// negative half
template <int DT, int STRIDE>
__device__ __forceinline__ int64_t digit32(const uint64_t* __restrict__ col, int i) {
  static_assert(DT == F32, "radix-2^16 split columns hold FP32 sums only");
  int64_t v = 0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int j = 2 * i + k;
    if (j < F32_R16_DIGITS)
      v += ((int64_t)col[j * STRIDE] - (int64_t)col[(F32_R16_DIGITS + j) * STRIDE]) * ((int64_t)1 << (16 * k));
  }
  return v;
}

#endif  // ES_F32_R32

// The exponent maximum as add_vec leaves it: one value, or for the FP32
// sign-split columns and the BF16 sign-split columns (pair-decoded) two
// 16-bit maxima packed in one word.
template <int DT, typename D>
__device__ __forceinline__ uint32_t emax_unpack(uint32_t e) {
  if constexpr (DT == F32 && sizeof(D) == 8 && D(-1) > D(0)) return max(e & 0xFFFFu, e >> 16);
#if ES_BF16_PACKED
  else if constexpr (DT == BF16 && sizeof(D) == 4 && D(-1) > D(0)) return max(e & 0xFFFFu, e >> 16);
#endif
  else return e;
}

// Additions between regularisations for a digit type.
template <int DT, typename D>
struct RegEvery {
  static constexpr int value = Geometry<DT>::REG_EVERY;
};
template <>
struct RegEvery<BF16, int32_t> {
  static constexpr int value = 60000;  // (2^31 - 2^7 - 2^23) / 2^15 > 65,000
};
template <>
struct RegEvery<BF16, uint32_t> {
  static constexpr int value = 120000;  // 255 + 120,000 * 2^15 < 2^32
};
template <>
struct RegEvery<F32, uint64_t> {
#if ES_F32_R32
  static constexpr int value = F32_R32_REG_EVERY;
#else
  static constexpr int value = 1 << 24;  // 2^16 + 2^24 * 2^39 < 2^64
#endif
};

// Classify one element for the special-value and signed-zero counters.
// flags bit 0: NaN, bit 1: +Inf, bit 2: -Inf, bit 3: not +0, bit 4: not -0.
template <int DT>
__device__ __forceinline__ uint32_t classify(uint64_t bits) {
  constexpr int W = Geometry<DT>::ELEM_BYTES * 8;
  constexpr int FB = DT == F64 ? 52 : (DT == F32 ? 23 : 7);
  constexpr uint64_t SIGN = (uint64_t)1 << (W - 1);
  constexpr uint64_t EXPM = (uint64_t)Geometry<DT>::EXP_SPECIAL << FB;
  constexpr uint64_t FRACM = ((uint64_t)1 << FB) - 1;
  uint32_t f = 0;
  if ((bits & EXPM) == EXPM) {
    if (bits & FRACM) f |= 1u;
    else f |= (bits & SIGN) ? 4u : 2u;
  }
  if (bits != 0) f |= 8u;
  if (bits != SIGN) f |= 16u;
  return f;
}

// Regularise a 72-digit radix-2^32 accumulator in place (one thread).
__device__ __forceinline__ void regularise72(int64_t* d) {
  int64_t carry = 0;
  for (int i = 0; i < ACC_DIGITS - 1; ++i) {
    const int64_t v = d[i] + carry;
    const int64_t c = (v + ((int64_t)1 << 31)) >> 32;
    d[i] = v - (c << 32);
    carry = c;
  }
  d[ACC_DIGITS - 1] += carry;
}

}  // namespace es
