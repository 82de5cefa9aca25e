// window.cuh -- the windowed tile reduction: one warp sums a contiguous
// range of elements exactly, keeping per lane only a small window of digits
// plus a warp-shared full-width overflow accumulator.  The segmented sum's
// windowed reducer (segmented.cu) runs it over its tile queue.
//
// Within one tile the exponents of real data are often concentrated
// (Section 6.3 notes that subtracting the mean leaves about 15 exponents in
// its Anderson-style dataset), so each lane keeps only WinGeom<DT>::WD
// digits below the largest digit of the tile's first batch (plus one carry
// digit), and any element that falls outside the window goes, exactly, into
// the warp's overflow accumulator in the format's native radix
// (shared-memory integer atomics).  The small columns let many more warps
// share an SM than the full 66-digit columns do.  Exact for every input;
// fast when most elements land in the window (Section 2: a sparse
// superaccumulator keeps only its active range of indices; here the
// inactive ones are not dropped, only slower).
#pragma once
#include <cstdint>

#include "digits.cuh"
#include "stream.cuh"

namespace es {

// Reducer shape per format: WD window digits per lane, W warps per CTA, U
// 16-byte vectors per lane per batch (two batches in flight).
#ifndef ES_WIN_F64_W
#define ES_WIN_F64_W 24
#endif
#ifndef ES_WIN_F64_U
#define ES_WIN_F64_U 4
#endif
template <int DT> struct WinGeom;
template <> struct WinGeom<F64> { static constexpr int WD = 4, W = ES_WIN_F64_W, U = ES_WIN_F64_U; };
#ifndef ES_WIN_N_W
#define ES_WIN_N_W 32
#endif
#ifndef ES_WIN_N_U
#define ES_WIN_N_U 2
#endif
template <> struct WinGeom<F32> { static constexpr int WD = 8, W = ES_WIN_N_W, U = ES_WIN_N_U; };
template <> struct WinGeom<BF16> { static constexpr int WD = 8, W = ES_WIN_N_W, U = ES_WIN_N_U; };

// Overflow adds per warp between regularisations of an FP64 overflow
// accumulator: each add changes a digit by at most 2^52, and a check comes
// at most one batch (32 lanes x 4 vectors x 2 elements) late.
constexpr int WIN_OVER_REG = 1024;

// Digit index of an element and its (signed) parts in the native radix.
template <int DT>
__device__ __forceinline__ void win_decode(uint64_t bits, int& d, int64_t& lo, int64_t& hi, uint32_t& E) {
  if constexpr (DT == F64) {
    const uint32_t lo32 = (uint32_t)bits, hi32 = (uint32_t)(bits >> 32);
    E = (hi32 >> 20) & 0x7FFu;
    const uint32_t mhi = (hi32 & 0xFFFFFu) | (E != 0u ? 0x100000u : 0u);
    const uint32_t p = max(E, 1u) - 1u;
    // sign applied before the shifts (see add_f64_e): for a negative
    // element the low digit gets 2^32 - (v mod 2^32), the high one ~(v >> 32)
    const uint32_t sm = (uint32_t)((int32_t)hi32 >> 31);
    const uint32_t xl = lo32 ^ sm, xh = mhi ^ sm;
    const uint32_t w0 = __funnelshift_l(sm, xl, p);
    const uint32_t w1 = __funnelshift_l(xl, xh, p);
    const uint32_t w2 = __funnelshift_l(xh, sm, p);
    lo = (int64_t)((uint64_t)w0 + (hi32 >> 31));
    hi = (int64_t)(((uint64_t)w2 << 32) | w1);
    d = (int)(p >> 5);
  } else {
    constexpr int FB = DT == F32 ? 23 : 7;
    constexpr uint32_t SIGN = DT == F32 ? 0x80000000u : 0x8000u;
    const uint32_t w = (uint32_t)bits;
    E = (w >> FB) & 0xFFu;
    const uint32_t m = (w & ((1u << FB) - 1u)) | (E != 0u ? (1u << FB) : 0u);
    const uint32_t p = max(E, 1u) - 1u;
    const int32_t sg = (w & SIGN) ? -1 : 0;
    lo = (int64_t)(((int32_t)(m << (p & 7u)) ^ sg) - sg);
    hi = 0;
    d = (int)(p >> 3);
  }
}

// Biased exponent field and native-radix digit index only (the window
// base scan needs no parts).
template <int DT>
__device__ __forceinline__ void win_digit(uint64_t bits, int& d, uint32_t& E) {
  if constexpr (DT == F64) {
    E = (uint32_t)(bits >> 52) & 0x7FFu;
    d = (int)((max(E, 1u) - 1u) >> 5);
  } else {
    E = ((uint32_t)bits >> (DT == F32 ? 23 : 7)) & 0xFFu;
    d = (int)((max(E, 1u) - 1u) >> 3);
  }
}

// Window column height (per lane) and overflow digits (per warp) of a format.
template <int DT>
__host__ __device__ constexpr int win_rows() { return WinGeom<DT>::WD + 1; }
template <int DT>
__host__ __device__ constexpr int win_over_digits() { return Geometry<DT>::DIGITS; }

// One warp (all 32 lanes) sums elements [elo, ehi) of x exactly.
//   cols: the CTA's window columns, digit-major with stride T (this lane's
//         column is cols + threadIdx.x, at least win_rows<DT>() rows);
//   ov:   this warp's overflow accumulator (win_over_digits<DT>() words).
// Both must be zero on entry and are zero again on return.  Out: d0, d1, d2
// = radix-2^32 words lane, lane + 32 and lane + 64 (0 for lane + 64 >=
// ACC_DIGITS) of the range's exact sum, carry-free; flags = the OR of the
// classification flags of the range's elements (see classify).
template <int DT, int T, int U>
__device__ __forceinline__ void win_tile(const void* x, int64_t elo, int64_t ehi, int64_t* cols, int64_t* ov,
                                         int64_t& d0, int64_t& d1, int64_t& d2, uint32_t& flags) {
  constexpr int WD = WinGeom<DT>::WD;
  constexpr int NC = WD + 1;                   // window column height (top digit takes carries)
  constexpr int ND = Geometry<DT>::DIGITS;     // overflow accumulator digits, native radix
  constexpr int RB = Geometry<DT>::RADIX_BITS;
  constexpr int EB = Geometry<DT>::ELEM_BYTES;
  constexpr int EPV = 16 / EB;
  constexpr int REG_EVERY = Geometry<DT>::REG_EVERY;
  constexpr int64_t PER = (int64_t)32 * U;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t* col = cols + threadIdx.x;
  auto decode = [&](uint64_t bits, int& d, int64_t& lo, int64_t& hi, uint32_t& E) {
    win_decode<DT>(bits, d, lo, hi, E);
  };
  const RangeSplit r = split_range<DT>(x, elo, ehi);
  const uint4* vp = reinterpret_cast<const uint4*>((const char*)x + r.vlo * EB);
  const int64_t cnt = (r.nvec > lane) ? (r.nvec - lane + 31) / 32 : 0;
  // full batches in which every lane has U vectors: warp-uniform, because
  // the loop below ends each batch with warp-collective operations
  const int64_t nb = r.nvec / PER;

  // ---- window base: the largest digit among the first batch of the tile ----
  uint4 A[U], B[U];
  // batch k (every lane has U vectors in it) into registers
  auto fetch = [&](int64_t k, uint4 (&R)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) R[u] = ldg_stream(vp + lane + k * PER + u * 32);
  };
  if (nb > 0) fetch(0, A);
  uint32_t etop = 0;
  {
    auto top_e = [&](uint64_t bits) {
      int d; uint32_t E;
      win_digit<DT>(bits, d, E);
      if (E != Geometry<DT>::EXP_SPECIAL) etop = max(etop, (uint32_t)d + 1u);
    };
    if (nb > 0) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t q[4] = {A[u].x, A[u].y, A[u].z, A[u].w};
        if constexpr (DT == F64) {
          top_e(((uint64_t)q[1] << 32) | q[0]);
          top_e(((uint64_t)q[3] << 32) | q[2]);
        } else if constexpr (DT == F32) {
          for (int k = 0; k < 4; ++k) top_e(q[k]);
        } else {
          for (int k = 0; k < 4; ++k) {
            top_e(q[k] & 0xFFFFu);
            top_e(q[k] >> 16);
          }
        }
      }
    } else {
      if (lane < r.head_n) top_e(load_one<DT>(x, r.vlo - r.head_n + lane));
      if (lane < r.tail_n) top_e(load_one<DT>(x, r.tail_lo + lane));
      if (lane < r.nvec)
        for (int e = 0; e < EPV; ++e) top_e(load_one<DT>(x, r.vlo + (int64_t)lane * EPV + e));
    }
  }
  etop = __reduce_max_sync(0xffffffffu, etop);  // top digit + 1 (0: nothing seen)
  // targets b .. b + WD - 1: FP64 elements need their digit and the one above
  const int b = (DT == F64) ? max((int)etop + 1 - WD, 0) : max((int)etop - WD, 0);

  uint32_t emax = 0;
  int reg_left = REG_EVERY;
  uint32_t nover = 0;  // this lane's overflow adds since the last check
  // one element into the window column or, exactly, into the overflow
  // accumulator; `track` updates the exponent maximum (the FP64 vector path
  // does that once per vector with a three-input maximum instead)
  auto add_bits_e = [&](uint64_t bits, bool track) {
    int d; int64_t lo, hi; uint32_t E;
    decode(bits, d, lo, hi, E);
    if (track) emax = max(emax, E);
    const unsigned rel = (unsigned)(d - b);
    if (rel <= (unsigned)(DT == F64 ? WD - 2 : WD - 1)) {
      col[rel * T] += lo;
      if constexpr (DT == F64) col[(rel + 1) * T] += hi;
    } else {
      atomicAdd((unsigned long long*)&ov[d], (unsigned long long)lo);
      if constexpr (DT == F64) atomicAdd((unsigned long long*)&ov[d + 1], (unsigned long long)hi);
      ++nover;
    }
  };
  auto add_bits = [&](uint64_t bits) { add_bits_e(bits, true); };
  auto add_vec_w = [&](const uint4& v) {
    if constexpr (DT == F64) {
      emax = __vimax3_u32(emax, (v.y >> 20) & 0x7FFu, (v.w >> 20) & 0x7FFu);
      add_bits_e(((uint64_t)v.y << 32) | v.x, false);
      add_bits_e(((uint64_t)v.w << 32) | v.z, false);
    } else if constexpr (DT == F32) {
      add_bits(v.x); add_bits(v.y); add_bits(v.z); add_bits(v.w);
    } else {
      add_bits(v.x & 0xFFFFu); add_bits(v.x >> 16); add_bits(v.y & 0xFFFFu); add_bits(v.y >> 16);
      add_bits(v.z & 0xFFFFu); add_bits(v.z >> 16); add_bits(v.w & 0xFFFFu); add_bits(v.w >> 16);
    }
  };
  // keep the window column and the FP64 overflow digits inside int64
  auto after_batch = [&](int adds) {
    reg_left -= adds;
    if (reg_left <= 0) {
      int64_t carry = 0;
      for (int i = 0; i < NC - 1; ++i) {
        const int64_t v = col[i * T] + carry;
        const int64_t c = (v + ((int64_t)1 << (RB - 1))) >> RB;
        col[i * T] = v - (c << RB);
        carry = c;
      }
      col[(NC - 1) * T] += carry;
      reg_left = REG_EVERY;
    }
    if constexpr (DT == F64) {
      const uint32_t warp_over = __reduce_add_sync(0xffffffffu, nover);
      if (warp_over >= (uint32_t)WIN_OVER_REG) {
        __syncwarp();
        if (lane == 0) regularise<DT, 1>(ov);
        __syncwarp();
        nover = 0;
      }
    }
  };

  if (lane < r.head_n) add_bits(load_one<DT>(x, r.vlo - r.head_n + lane));
  for (int64_t k = 0; k < nb; k += 2) {
    if (k + 1 < nb) fetch(k + 1, B);
#pragma unroll
    for (int u = 0; u < U; ++u) add_vec_w(A[u]);
    after_batch(U * EPV);
    if (k + 1 >= nb) break;
    if (k + 2 < nb) fetch(k + 2, A);
#pragma unroll
    for (int u = 0; u < U; ++u) add_vec_w(B[u]);
    after_batch(U * EPV);
  }
  for (int64_t j = nb * U; j < cnt; ++j) add_vec_w(ldg_stream(vp + lane + j * 32));
  if (lane < r.tail_n) add_bits(load_one<DT>(x, r.tail_lo + lane));
  after_batch(REG_EVERY);  // forces the window regularisation before the merge
  // the overflow digits too: the merge below shifts narrow-format digits by
  // up to 24 bits, so they must be small
  __syncwarp();
  if (lane == 0) regularise<DT, 1>(ov);

  flags = 24u;
  if (emax == Geometry<DT>::EXP_SPECIAL || emax == 0u) flags = rescan_split<DT, 32>(x, r, lane);
  flags = __reduce_or_sync(0xffffffffu, flags);
  __syncwarp();

  // ---- merge: window columns at offset b plus the overflow accumulator ----
  const int64_t* wcols = cols + warp * 32;
  auto native = [&](int n) -> int64_t {  // native-radix digit n of the warp's sum
    int64_t v = (n < ND) ? ov[n] : 0;
    const int rel = n - b;
    if (rel >= 0 && rel < NC) {
#pragma unroll 8
      for (int k = 0; k < 32; ++k) v += wcols[rel * T + ((k + lane) & 31)];
    }
    return v;
  };
  auto word = [&](int i) -> int64_t {  // radix-2^32 word i
    if constexpr (DT == F64) {
      return native(i);
    } else {
      int64_t v = 0;
      for (int j = 0; j < 4; ++j) v += native(4 * i + j) * ((int64_t)1 << (8 * j));
      return v;
    }
  };
  d0 = word(lane);
  d1 = word(lane + 32);
  d2 = (lane + 64 < ACC_DIGITS) ? word(lane + 64) : 0;
  __syncwarp();
  for (int i = 0; i < NC; ++i) col[i * T] = 0;
  for (int i = lane; i < ND; i += 32) ov[i] = 0;
  __syncwarp();
}

}  // namespace es
