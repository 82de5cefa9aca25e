// finalize.cuh -- signed-carry propagation and the single rounding step.
//
// Section 3 step 6 / Section 5 step 4: turn the regularised, overlapping
// digits into a non-overlapping representation by propagating the signed
// carries once.  Here the digits are radix-2^32 signed 64-bit integers and
// the non-overlapping form is a two's-complement number in 32-bit limbs,
// then sign and magnitude.
//
// Section 3 step 7 / Section 5 step 5: locate the most significant non-zero
// bit, keep the target precision and round the rest by the mode.  Round to
// nearest-even is the default; it is always faithful in the sense of the
// problem statement (Section 1).  Subnormal results, overflow and the
// special-value rules of the library are handled here.
#pragma once
#include <cstdint>

#include "digits.cuh"

namespace es {

struct OutFormat {
  int frac_bits, exp_bits, bias, width;
};

__device__ __forceinline__ OutFormat out_format(int dt) {
  if (dt == F64) return {52, 11, 1023, 8};
  if (dt == F32) return {23, 8, 127, 4};
  return {7, 8, 127, 2};
}

// bits [pos, pos + 64) of the magnitude held in `nl` little-endian limbs
// (positions outside [0, 32 nl) read as zero; pos may be negative)
__device__ __forceinline__ uint64_t limb_window(const uint32_t* m, int nl, int pos) {
  const int li = (pos >= 0) ? (pos >> 5) : -((-pos + 31) >> 5);
  const int sh = pos - 32 * li;  // 0..31
  uint32_t a[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int j = li + k;
    a[k] = (j >= 0 && j < nl) ? m[j] : 0u;
  }
  const uint32_t lo = __funnelshift_r(a[0], a[1], sh);
  const uint32_t hi = __funnelshift_r(a[1], a[2], sh);
  return ((uint64_t)hi << 32) | lo;
}

// is any bit in [0, pos) set?
__device__ __forceinline__ bool any_below(const uint32_t* m, int nl, int pos) {
  if (pos <= 0) return false;
  const int full = min(pos >> 5, nl);
  for (int j = 0; j < full; ++j)
    if (m[j]) return true;
  const int rem = pos & 31;
  if (rem && (pos >> 5) < nl) return (m[pos >> 5] & ((1u << rem) - 1u)) != 0u;
  return false;
}

__device__ __forceinline__ uint64_t encode(const OutFormat& f, uint32_t sign, uint64_t biased,
                                           uint64_t frac) {
  return ((uint64_t)sign << (8 * f.width - 1)) | (biased << f.frac_bits) | frac;
}

// Round (-1)^sign * M * 2^unit_exp, M > 0 with bit length L, into format
// `out` under `mode`.
static __device__ uint64_t round_magnitude(const uint32_t* m, int nl, int L, uint32_t sign, int unit_exp,
                                   int out, int mode) {
  const OutFormat f = out_format(out);
  const int P = f.frac_bits + 1;
  const int emin = 1 - f.bias, emax = f.bias;
  const int e = L - 1 + unit_exp;                  // exponent of the leading bit
  int qexp = max(e, emin) - (P - 1);               // exponent of the last kept bit
  const int shift = qexp - unit_exp;               // number of dropped low bits
  uint64_t q;
  bool up = false;
  if (shift <= 0) {
    q = limb_window(m, nl, 0) << (-shift);         // exact (M < 2^P here)
  } else {
    q = limb_window(m, nl, shift);                 // bits above L are zero
    const bool half = (limb_window(m, nl, shift - 1) & 1u) != 0;
    const bool sticky = any_below(m, nl, shift - 1);
    const bool inexact = half || sticky;
    if (mode == RNE) up = half && (sticky || (q & 1u));
    else if (mode == RUP) up = inexact && !sign;
    else if (mode == RDOWN) up = inexact && sign;
  }
  q += up ? 1u : 0u;
  if (q == ((uint64_t)1 << P)) {
    q >>= 1;
    qexp += 1;
  }
  if (qexp + (P - 1) > emax) {
    bool to_inf = (mode == RNE) || (mode == RUP && !sign) || (mode == RDOWN && sign);
    if (to_inf) return encode(f, sign, ((uint64_t)1 << f.exp_bits) - 1, 0);
    return encode(f, sign, ((uint64_t)1 << f.exp_bits) - 2, ((uint64_t)1 << f.frac_bits) - 1);
  }
  if (q < ((uint64_t)1 << (P - 1))) return encode(f, sign, 0, q);  // subnormal
  return encode(f, sign, (uint64_t)(qexp + (P - 1) + f.bias), q - ((uint64_t)1 << (P - 1)));
}

// Result bits for an accumulator (ACC_WORDS words; digits need not be
// regularised as long as |digit| < 2^62).  `limbs` is scratch for
// ACC_DIGITS words.  One thread.
static __device__ uint64_t finalize_acc(const int64_t* acc, uint32_t* limbs, int in_dt, int out,
                                 int mode) {
  const OutFormat f = out_format(out);
  const uint64_t sign_bit = (uint64_t)1 << (8 * f.width - 1);
  const uint64_t inf = encode(f, 0, ((uint64_t)1 << f.exp_bits) - 1, 0);
  if (acc[W_COUNT] == 0) return 0;                                     // empty: +0
  if (acc[W_NAN] || (acc[W_PINF] && acc[W_NINF]))
    return inf | ((uint64_t)1 << (f.frac_bits - 1));                   // quiet NaN
  if (acc[W_PINF]) return inf;
  if (acc[W_NINF]) return inf | sign_bit;
  // signed-carry propagation into 32-bit two's-complement limbs
  int64_t carry = 0;
  for (int i = 0; i < ACC_DIGITS; ++i) {
    const int64_t t = acc[i] + carry;
    limbs[i] = (uint32_t)t;
    carry = t >> 32;
  }
  const uint32_t sign = carry < 0 ? 1u : 0u;
  if (sign) {  // magnitude = two's-complement negation
    uint64_t c = 1;
    for (int i = 0; i < ACC_DIGITS; ++i) {
      const uint64_t t = (uint64_t)(uint32_t)~limbs[i] + c;
      limbs[i] = (uint32_t)t;
      c = t >> 32;
    }
  }
  int top = ACC_DIGITS - 1;
  while (top >= 0 && limbs[top] == 0u) --top;
  if (top < 0) {  // exact zero
    if (acc[W_NOTNZ] == 0) return sign_bit;  // every input was -0
    if (acc[W_NOTPZ] == 0) return 0;         // every input was +0
    return mode == RDOWN ? sign_bit : 0;
  }
  const int L = 32 * top + (32 - __clz(limbs[top]));
  return round_magnitude(limbs, top + 1, L, sign, unit_exp_of(in_dt), out, mode);
}

__device__ __forceinline__ void store_result(void* dst, int out, uint64_t bits) {
  if (out == F64) *(unsigned long long*)dst = bits;
  else if (out == F32) *(uint32_t*)dst = (uint32_t)bits;
  else *(uint16_t*)dst = (uint16_t)bits;
}

}  // namespace es
