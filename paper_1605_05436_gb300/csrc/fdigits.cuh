// fdigits.cuh -- BF16 superaccumulator digits added on the FP32 FMA pipe.
//
// Section 2 allows the components of a superaccumulator to be floating-point
// numbers as long as every addition into them is exact.  A BF16 element has
// only 8 significant bits, so a digit column of FP32 numbers can take many of
// them exactly:
//
//   digit i (i = E >> 3, E the biased exponent, 32 digits) collects the
//   elements with E in [8i, 8i + 7], each scaled by 2^(127 - 8i):
//       d = x * 2^(127 - 8i) = (-1)^s * m * 2^(E - 8i - 7)
//   with m = 2^7 + F for E >= 1 (for E = 0, x * 2^127 = (-1)^s * 2F * 2^-7,
//   the same formula with m = 2F), so every d is a multiple of 2^-7 with
//   |d| <= 255.  A sum of k such values is a multiple of 2^-7 below
//   255 k, which FP32 holds exactly while 255 k < 2^17 (24 significant bits
//   from 2^-7 up): k <= 514 additions per digit between flushes.  One FFMA
//   does the scaling and the addition (the product is exact, and the sum
//   is exact by the bound, so its single rounding changes nothing).
//
// The scale 2^(127 - 8i) is built from the bits: its exponent field is
// 254 - 8i, i.e. the word 0x7F000000 - (i << 26), and i << 26 is the
// element's exponent bits 10-14 moved to bits 26-30.  Specials (E = 255)
// land in digit 31 as an infinity or NaN and are detected at the flush.
//
// Flush (every <= 514 additions): each FP32 digit times 2^7 is an integer
// D below 2^24 in magnitude; it is added into an int32 digit of radix 2^8
// whose unit is 2^-134 (half the BF16 smallest subnormal: the value of an
// element in these units, m * 2^(E - 8i) at digit i, is always even, so the
// whole sum is too, and the CTA merge halves it exactly).  The int32 digits
// are regularised (Lemma 1, balanced carries to the neighbour) every
// FDIG_REG_FLUSHES flushes, before any can overflow.
#pragma once
#include <cstdint>

#include "digits.cuh"

namespace es {

#ifndef ES_BF16F_PAIR
#define ES_BF16F_PAIR 0
#endif

constexpr int FDIG_DIGITS = 32;          // FP32 digits per thread
constexpr int FDIG_INT_DIGITS = 33;      // int32 radix-2^8 digits per thread (digit 32: carries)
constexpr int FDIG_MAX_ADDS = 514;       // exact additions per FP32 digit between flushes
constexpr int FDIG_REG_FLUSHES = 64;     // flushes between int32 regularisations:
                                         // 2^8 + 64 * 2^24 < 2^31

// The two elements of a 32-bit word (low half first) into the FP32 digit
// column `fc` (digit stride STRIDE floats).
// Digit i sits i * STRIDE floats = i * 4 * STRIDE bytes after digit 0; with
// STRIDE a multiple of 256 that is (i << 10) * (STRIDE / 256) bytes, so the
// masked exponent bits give the address with one multiply-add.
// (Other strides: the digit index is shifted down first.)
template <int STRIDE>
__device__ __forceinline__ void fdig_add_pair(float* __restrict__ fc, uint32_t w) {
  const uint32_t a0 = w & 0x00007C00u;           // (E0 >> 3) << 10
  const uint32_t a1 = w & 0x7C000000u;           // (E1 >> 3) << 26
  const float x0 = __uint_as_float(w << 16);
  const float x1 = __uint_as_float(w & 0xFFFF0000u);
  const float s0 = __uint_as_float(0x7F000000u - (a0 << 16));
  const float s1 = __uint_as_float(0x7F000000u - a1);
  float* d0;
  float* d1;
  if constexpr (STRIDE % 256 == 0) {
    d0 = (float*)((char*)fc + a0 * (uint32_t)(STRIDE / 256));
    d1 = (float*)((char*)fc + (a1 >> 16) * (uint32_t)(STRIDE / 256));
  } else {
    // (a multiply-high of the shifted exponent bits, one FMA-pipe
    // instruction instead of a shift and a multiply-add, measured 10% slower)
    d0 = fc + (a0 >> 10) * STRIDE;
    d1 = fc + (a1 >> 26) * STRIDE;
  }
#if ES_BF16F_PAIR
  // both digits read before either is written, so the two additions do not
  // wait on each other; when both elements fall in one digit, the upper
  // element adds onto the lower one's result (and its store comes last)
  const float v0 = *d0;
  const float v1 = *d1;
  const float r0 = __fmaf_rn(x0, s0, v0);
  const float r1 = __fmaf_rn(x1, s1, d0 == d1 ? r0 : v1);
  *d0 = r0;
  *d1 = r1;
#else
  *d0 = __fmaf_rn(x0, s0, *d0);
  *d1 = __fmaf_rn(x1, s1, *d1);
#endif
}

#ifndef ES_BF16F_ADDR
#define ES_BF16F_ADDR 0
#endif

// The same with the digit addresses as 32-bit shared-memory offsets, both
// formed by one multiply-add on the FMA pipe (the upper element's by the
// high half of a product: (a1 >> 16) * c = hi(a1 * (c << 16)) since the low
// 16 bits of a1 are zero).  `fbase` is the shared-memory address of digit 0.
template <int STRIDE>
__device__ __forceinline__ void fdig_add_pair_s(uint32_t fbase, uint32_t w) {
  static_assert(STRIDE % 256 == 0, "digit stride must be a multiple of 256 floats");
  constexpr uint32_t C = STRIDE / 256;
  const uint32_t a0 = w & 0x00007C00u;
  const uint32_t a1 = w & 0x7C000000u;
  uint32_t p0, p1;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(p0) : "r"(a0), "n"(C), "r"(fbase));
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(p1) : "r"(a1), "n"(C << 16), "r"(fbase));
  const float x0 = __uint_as_float(w << 16);
  const float x1 = __uint_as_float(w & 0xFFFF0000u);
  const float s0 = __uint_as_float(0x7F000000u - (a0 << 16));
  const float s1 = __uint_as_float(0x7F000000u - a1);
  float v0, v1;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v0) : "r"(p0) : "memory");
  v0 = __fmaf_rn(x0, s0, v0);
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(p0), "f"(v0) : "memory");
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v1) : "r"(p1) : "memory");
  v1 = __fmaf_rn(x1, s1, v1);
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(p1), "f"(v1) : "memory");
}

// Two digit sets: the lower element of each word into set 0, the upper one
// into set 1 (distinct arrays, so the two read-modify-writes are independent).
template <int STRIDE>
__device__ __forceinline__ void fdig_add_pair2(float* __restrict__ f0, float* __restrict__ f1, uint32_t w) {
  const uint32_t a0 = w & 0x00007C00u;
  const uint32_t a1 = w & 0x7C000000u;
  const float x0 = __uint_as_float(w << 16);
  const float x1 = __uint_as_float(w & 0xFFFF0000u);
  const float s0 = __uint_as_float(0x7F000000u - (a0 << 16));
  const float s1 = __uint_as_float(0x7F000000u - a1);
  float* d0 = (float*)((char*)f0 + a0 * (uint32_t)(STRIDE / 256));
  float* d1 = (float*)((char*)f1 + (a1 >> 16) * (uint32_t)(STRIDE / 256));
  const float v0 = *d0, v1 = *d1;
  *d0 = __fmaf_rn(x0, s0, v0);
  *d1 = __fmaf_rn(x1, s1, v1);
}

template <int STRIDE>
__device__ __forceinline__ void fdig_add_vec2(float* __restrict__ f0, float* __restrict__ f1, const uint4& v) {
  fdig_add_pair2<STRIDE>(f0, f1, v.x);
  fdig_add_pair2<STRIDE>(f0, f1, v.y);
  fdig_add_pair2<STRIDE>(f0, f1, v.z);
  fdig_add_pair2<STRIDE>(f0, f1, v.w);
}

// One element (h < 2^16).
template <int STRIDE>
__device__ __forceinline__ void fdig_add_one(float* __restrict__ fc, uint32_t h) {
  const uint32_t a = h & 0x7C00u;
  const float x = __uint_as_float(h << 16);
  const float s = __uint_as_float(0x7F000000u - (a << 16));
  float* d = fc + (a >> 10) * STRIDE;  // (cold path)
  *d = __fmaf_rn(x, s, *d);
}

template <int STRIDE>
__device__ __forceinline__ void fdig_add_vec(float* __restrict__ fc, const uint4& v) {
#if ES_BF16F_ADDR
  const uint32_t fb = (uint32_t)__cvta_generic_to_shared(fc);
  fdig_add_pair_s<STRIDE>(fb, v.x);
  fdig_add_pair_s<STRIDE>(fb, v.y);
  fdig_add_pair_s<STRIDE>(fb, v.z);
  fdig_add_pair_s<STRIDE>(fb, v.w);
#else
  fdig_add_pair<STRIDE>(fc, v.x);
  fdig_add_pair<STRIDE>(fc, v.y);
  fdig_add_pair<STRIDE>(fc, v.z);
  fdig_add_pair<STRIDE>(fc, v.w);
#endif
}

// Balanced regularisation of the int32 digits (|D| <= 2^7 afterwards,
// except the top digit, which takes the last carry).
template <int STRIDE>
__device__ __forceinline__ void fdig_regularise(int32_t* __restrict__ ic) {
  int32_t carry = 0;
#pragma unroll 4
  for (int i = 0; i < FDIG_INT_DIGITS - 1; ++i) {
    const int32_t v = ic[i * STRIDE] + carry;
    const int32_t c = (v + 128) >> 8;
    ic[i * STRIDE] = v - (c << 8);
    carry = c;
  }
  ic[(FDIG_INT_DIGITS - 1) * STRIDE] += carry;
}

// Move the FP32 digits into the int32 digits and clear them.  `spec` keeps
// the largest exponent field seen in a digit: 0x7F800000 means a digit held
// an infinity or NaN (an element with E = 255 was added).
template <int STRIDE>
__device__ __forceinline__ void fdig_flush(float* __restrict__ fc, int32_t* __restrict__ ic, uint32_t& spec) {
#pragma unroll 8
  for (int i = 0; i < FDIG_DIGITS; ++i) {
    const float v = fc[i * STRIDE];
    fc[i * STRIDE] = 0.0f;
    spec = max(spec, __float_as_uint(v) & 0x7F800000u);
    // exact: v is a multiple of 2^-7 below 2^17 (for a non-finite v the
    // integer is meaningless, and the special-value rules decide the result)
    const int32_t D = __float2int_rn(v * 128.0f);
    ic[i * STRIDE] = (int32_t)((uint32_t)ic[i * STRIDE] + (uint32_t)D);
  }
}

// The same flush into int32 digits held in registers (I[0..32], the loops
// fully unrolled so that every index is static).
template <int STRIDE>
__device__ __forceinline__ void fdig_flush_regs(float* __restrict__ fc, int32_t (&I)[FDIG_INT_DIGITS],
                                                uint32_t& spec) {
#pragma unroll
  for (int i = 0; i < FDIG_DIGITS; ++i) {
    const float v = fc[i * STRIDE];
    fc[i * STRIDE] = 0.0f;
    spec = max(spec, __float_as_uint(v) & 0x7F800000u);
    I[i] = (int32_t)((uint32_t)I[i] + (uint32_t)__float2int_rn(v * 128.0f));
  }
}

// Warp-transposed flush: lane j takes FP32 digit j of every lane of its warp
// (columns read rotated by lane, so no two lanes hit one bank), adds them
// into its own int64 `wd` -- digit j of the warp's radix-2^8 accumulator in
// half units -- and clears them.  32 lanes x |D| < 2^24 per flush: an int64
// digit never needs a carry.  `wcols` is this warp's first column.
template <int STRIDE>
__device__ __forceinline__ void fdig_flush_warp(float* __restrict__ wcols, int lane, int64_t& wd, uint32_t& spec) {
  __syncwarp();
  float* row = wcols + lane * STRIDE;
#pragma unroll 8
  for (int l = 0; l < 32; ++l) {
    const int c = (l + lane) & 31;
    const float v = row[c];
    row[c] = 0.0f;
    spec = max(spec, __float_as_uint(v) & 0x7F800000u);
    wd += (int64_t)__float2int_rn(v * 128.0f);
  }
  __syncwarp();
}

__device__ __forceinline__ void fdig_regularise_regs(int32_t (&I)[FDIG_INT_DIGITS]) {
  int32_t carry = 0;
#pragma unroll
  for (int i = 0; i < FDIG_INT_DIGITS - 1; ++i) {
    const int32_t v = I[i] + carry;
    const int32_t c = (v + 128) >> 8;
    I[i] = v - (c << 8);
    carry = c;
  }
  I[FDIG_INT_DIGITS - 1] += carry;
}

}  // namespace es
