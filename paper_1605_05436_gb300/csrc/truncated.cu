// truncated.cu -- the condition-number-sensitive sum (Section 4, the r <- r^2
// iteration over r-truncated sparse superaccumulators; Section 2, sparse and
// gamma-truncated superaccumulators).
//
// One pass with truncation parameter R:
//   1. every thread keeps a window of the R most significant radix-2^32
//      digits of its running sum in shared memory (the r-truncated sparse
//      superaccumulator of its chain of additions: a left-deep summation
//      tree).  An element is split into two digit parts; a part above the
//      window moves the window up (the digits that fall out of the bottom are
//      dropped), a part below the window is dropped;
//   2. every non-zero dropped item is counted.  Each lies at a digit at or
//      below the bottom of its thread's final window (the window only moves
//      up), maxdrop = the highest such bottom over the threads that dropped
//      anything; a dropped element part at digit j is smaller than
//      2^(32j + 52) units, a dropped window digit (regularised first) smaller
//      than 2^(32j + 32), so the total truncated mass is at most
//      B = events * 2^(32 * maxdrop + 52) units;
//   3. the threads' windows are merged exactly (CTA, then the last CTA over
//      the CTAs' partials) into S, the sum of the truncated chains;
//   4. stopping condition: the last CTA rounds S - B, S and S + B; when the
//      three agree, every value within B of S -- the exact sum among them --
//      rounds to the same result, which is returned and the iteration stops.
//      This is the paper's test that the result is unchanged by adding or
//      subtracting a bound of everything truncated, taken on the unrounded
//      sum so that the result is the correctly rounded exact sum.
// The host runs R = 2, 4, 16 (r <- r^2 from r = 2) and, when R reaches the
// digits a format can occupy (67 for FP64, 10 for FP32, 9 for BF16), the
// exact single-pass kernel, which is the untruncated case.
#include <cuda_runtime.h>

#include <atomic>

#include <cstring>

#include "../../include/exactsum.h"
#include "digits.cuh"
#include "finalize.cuh"
#include "handle.h"
#include "internal.h"
#include "stream.cuh"

namespace es {

struct TruncArgs {
  const void* x;
  int64_t n, head, nvec, tail;
  int out, mode;
  void* result;
  int64_t* partials;             // grid x ACC_WORDS
  unsigned int* ticket;          // zero between launches; reset by the last CTA
  unsigned long long* state;     // [0] events, [1] highest dropped digit + 1, [2] stop (zeroed by the host)
};

#ifndef ES_TR_T
#define ES_TR_T 1024
#endif
constexpr int TR_T = ES_TR_T;  // threads per CTA (1,024: 2^28 uniform input 0.99 ms for its two
                               // passes, 768: 1.07 ms, 512: 1.37 ms)
#ifndef ES_TR_U
#define ES_TR_U 2
#endif
constexpr int TR_U = ES_TR_U;  // 16-byte vectors per thread per batch (two batches in flight)
constexpr int TR_REG_EVERY = 1984;  // digit parts between window regularisations (each < 2^52)

// An element as two radix-2^32 digit parts: value = lo * 2^(32k) + hi * 2^(32(k+1))
// units, lo in [0, 2^32], hi in [-2^52, 2^52) (the sign folded as in add_f64_e).
// E is the element's biased exponent field.
template <int DT>
__device__ __forceinline__ void split32(uint64_t bits, uint32_t E, int& k, int64_t& lo, int64_t& hi) {
  uint32_t mlo, mhi, neg;
  if constexpr (DT == F64) {
    const uint32_t h = (uint32_t)(bits >> 32);
    mlo = (uint32_t)bits;
    mhi = (h & 0xFFFFFu) | (E != 0u ? 0x100000u : 0u);
    neg = h >> 31;
  } else if constexpr (DT == F32) {
    const uint32_t w = (uint32_t)bits;
    mlo = (w & 0x7FFFFFu) | (E != 0u ? 0x800000u : 0u);
    mhi = 0;
    neg = w >> 31;
  } else {
    const uint32_t w = (uint32_t)bits & 0xFFFFu;
    mlo = (w & 0x7Fu) | (E != 0u ? 0x80u : 0u);
    mhi = 0;
    neg = w >> 15;
  }
  const uint32_t p = max(E, 1u) - 1u;
  const uint32_t sm = 0u - neg;
  const uint32_t xl = mlo ^ sm, xh = mhi ^ sm;
  const uint32_t w0 = __funnelshift_l(sm, xl, p);
  const uint32_t w1 = __funnelshift_l(xl, xh, p);
  const uint32_t w2 = __funnelshift_l(xh, sm, p);
  k = (int)(p >> 5);
  lo = (int64_t)((uint64_t)w0 + neg);
  hi = (int64_t)(((uint64_t)w2 << 32) | w1);
}

// The R-digit window of one thread: slot s (0 <= s < R) holds digit
// low + 1 + s, top = low + R (slot s at col[s * TR_T]).  Digits at or below
// `low` are outside the window; `low` never decreases, so every item a
// thread drops lies at a digit <= its final `low`.
//
// The rare window moves are kept out of line (so that the per-element path
// stays small) and report what they did packed into one 64-bit value:
// new top | (non-zero digits dropped) << 32.
__device__ __forceinline__ uint64_t win_pack(int top, uint32_t dropped) {
  return (uint64_t)(uint32_t)top | ((uint64_t)dropped << 32);
}

// Move the window up by d >= 1 digits: slots below d leave (counted when
// non-zero), the rest move down, the top d slots start at zero.
template <int R>
__device__ __forceinline__ uint32_t win_shift(int64_t* col, int d) {
  uint32_t dropped = 0;
#pragma unroll 1
  for (int s = 0; s < R; ++s) {
    int64_t& v = col[s * TR_T];
    if (s < d && v != 0) ++dropped;
    v = s + d < R ? col[(s + d) * TR_T] : 0;
  }
  return dropped;
}

// Lemma 1 carries inside the window (balanced digits); a carry out of the
// top digit moves the window up by one.
template <int R>
__device__ __noinline__ uint64_t win_regularise(int64_t* col, int top) {
  uint32_t dropped = 0;
  int64_t carry = 0;
#pragma unroll 1
  for (int s = 0; s < R; ++s) {
    const int64_t v = col[s * TR_T] + carry;
    const int64_t c = (v + ((int64_t)1 << 31)) >> 32;
    col[s * TR_T] = v - (c << 32);
    carry = c;
  }
  if (carry != 0) {
    dropped = win_shift<R>(col, 1);
    col[(R - 1) * TR_T] = carry;
    ++top;
  }
  return win_pack(top, dropped);
}

// Move the window up so that its top digit is t (> top), regularising first.
template <int R>
__device__ __noinline__ uint64_t win_raise(int64_t* col, int top, int t) {
  const uint64_t rg = win_regularise<R>(col, top);
  top = (int)(uint32_t)rg;
  uint32_t dropped = (uint32_t)(rg >> 32);
  if (t > top) {
    dropped += win_shift<R>(col, t - top < R ? t - top : R);
    top = t;
  }
  return win_pack(top, dropped);
}

template <int R>
struct Window {
  int64_t* col;
  int top;                     // most significant digit held; -1 while empty
  int low;                     // top - R
  unsigned long long events;   // non-zero items dropped
  int adds;                    // parts added since the last regularisation

  __device__ __forceinline__ int64_t& slot(int s) { return col[s * TR_T]; }

  __device__ __forceinline__ void absorb(uint64_t r) {
    top = (int)(uint32_t)r;
    low = top - R;
    events += r >> 32;
  }

  __device__ __forceinline__ void regularise() {
    adds = 0;
    if (top >= 0) absorb(win_regularise<R>(col, top));
  }

  // Add an element's parts: lo at digit k, hi at digit k + 1, u = k - low - 1
  // the slot of the lo part.
  //  - both inside (0 <= u <= R - 2): two slot additions, one unsigned compare;
  //  - below (u < 0): the lo part is dropped, and so is the hi part unless
  //    u = -1 (then it goes to slot 0); non-zero dropped parts are counted;
  //  - at or above the top: the window moves up first when a non-zero part
  //    lies above it (out of line: rare once the largest magnitudes have
  //    been seen); afterwards u is R - 2, or R - 1 with hi = 0.
  // (A warp vote so that all lanes take one path measured 3 % faster on ill-
  // conditioned input and 6 % slower on well-conditioned input.)
  __device__ __forceinline__ void add_pair(int k, int64_t lo, int64_t hi) {
    int u = k - low - 1;
    if ((unsigned)u <= (unsigned)(R - 2)) {
      slot(u) += lo;
      slot(u + 1) += hi;
    } else if (u < 0) {
      if (u == -1) slot(0) += hi;
      events += (unsigned)(lo != 0) + (unsigned)(u < -1 && hi != 0);
    } else {
      const int t = hi != 0 ? k + 1 : k;
      if (t > top) {
        if (top < 0) {
          top = t;
          low = top - R;
        } else {
          absorb(win_raise<R>(col, top, t));
        }
        u = k - low - 1;
      }
      slot(u) += lo;
      if (u + 1 < R) slot(u + 1) += hi;
    }
  }

  // once per vector: every lane counts alike, so that lanes regularise
  // together (a window move regularises too but does not reset the count)
  __device__ __forceinline__ void tick(int parts) {
    adds += parts;
    if (adds >= TR_REG_EVERY) regularise();
  }
};

template <int DT, int R>
__device__ __forceinline__ void add_elem(Window<R>& w, uint64_t bits, uint32_t E) {
  int k;
  int64_t lo, hi;
  split32<DT>(bits, E, k, lo, hi);
  w.add_pair(k, lo, hi);
}

// All elements of one 16-byte vector; the exponent maximum by three-input
// maxima, once per two exponents.
template <int DT, int R>
__device__ __forceinline__ void add_vec16(Window<R>& w, const uint4& v, uint32_t& emax) {
  if constexpr (DT == F64) {
    const uint32_t e0 = (v.y >> 20) & 0x7FFu, e1 = (v.w >> 20) & 0x7FFu;
    emax = __vimax3_u32(emax, e0, e1);
    add_elem<DT, R>(w, ((uint64_t)v.y << 32) | v.x, e0);
    add_elem<DT, R>(w, ((uint64_t)v.w << 32) | v.z, e1);
    w.tick(4);
  } else if constexpr (DT == F32) {
    const uint32_t q[4] = {v.x, v.y, v.z, v.w};
    uint32_t e[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) e[j] = (q[j] >> 23) & 0xFFu;
    emax = __vimax3_u32(emax, e[0], e[1]);
    emax = __vimax3_u32(emax, e[2], e[3]);
#pragma unroll
    for (int j = 0; j < 4; ++j) add_elem<DT, R>(w, q[j], e[j]);
    w.tick(8);
  } else {
    const uint32_t q[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t e0 = (q[j] >> 7) & 0xFFu, e1 = (q[j] >> 23) & 0xFFu;
      emax = __vimax3_u32(emax, e0, e1);
      add_elem<DT, R>(w, q[j] & 0xFFFFu, e0);
      add_elem<DT, R>(w, q[j] >> 16, e1);
    }
    w.tick(16);
  }
}

// One element outside the vectors (head or tail).
template <int DT, int R>
__device__ __forceinline__ void add_one_elem(Window<R>& w, uint64_t bits, uint32_t& emax) {
  constexpr int FB = DT == F64 ? 52 : (DT == F32 ? 23 : 7);
  const uint32_t E = (uint32_t)((bits >> FB) & (uint64_t)Geometry<DT>::EXP_SPECIAL);
  emax = max(emax, E);
  add_elem<DT, R>(w, bits, E);
  w.tick(2);
}

template <int DT, int R>
__global__ void __launch_bounds__(TR_T, 1) trunc_sum_kernel(TruncArgs a) {
  constexpr int EB = Geometry<DT>::ELEM_BYTES;
  constexpr int EPV = 16 / EB;
  constexpr int NW = TR_T / 32;
  extern __shared__ int64_t tr_cols[];  // R x TR_T
  __shared__ int tops[TR_T];
  __shared__ int64_t blk[ACC_WORDS];
  __shared__ int64_t tmp[ACC_WORDS];
  __shared__ uint32_t limbs[ACC_DIGITS];
  __shared__ uint32_t blk_flags, is_last;
  __shared__ unsigned long long blk_events;
  __shared__ int blk_maxdrop;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t G = gridDim.x;
  if (t == 0) {
    blk_flags = 0;
    blk_events = 0;
    blk_maxdrop = -1;
  }
  Window<R> w;
  w.col = tr_cols + t;
  w.top = -1;
  w.low = -1 - R;
  w.events = 0;
  w.adds = 0;
#pragma unroll
  for (int s = 0; s < R; ++s) w.col[s * TR_T] = 0;

  // this thread's vectors vb + t + j*T (the same ownership as the exact kernel)
  const uint4* vx = reinterpret_cast<const uint4*>((const char*)a.x + a.head * EB);
  const int64_t vb = a.nvec * blockIdx.x / G, ve = a.nvec * (blockIdx.x + 1) / G;
  uint32_t emax = 0;
  const int64_t cnt = (vb + t < ve) ? (ve - vb - t + TR_T - 1) / TR_T : 0;
  const uint4* p = vx + vb + t;
  const int64_t nb = cnt / TR_U;
  // two batches in flight: the next batch loads while this one is added
  uint4 A[TR_U], B[TR_U];
  if (nb > 0) {
#pragma unroll
    for (int u = 0; u < TR_U; ++u) A[u] = ldg_stream(p + u * TR_T);
  }
  for (int64_t k = 0; k < nb; k += 2) {
    if (k + 1 < nb) {
#pragma unroll
      for (int u = 0; u < TR_U; ++u) B[u] = ldg_stream(p + ((k + 1) * TR_U + u) * TR_T);
    }
#pragma unroll
    for (int u = 0; u < TR_U; ++u) add_vec16<DT, R>(w, A[u], emax);
    if (k + 1 >= nb) break;
    if (k + 2 < nb) {
#pragma unroll
      for (int u = 0; u < TR_U; ++u) A[u] = ldg_stream(p + ((k + 2) * TR_U + u) * TR_T);
    }
#pragma unroll
    for (int u = 0; u < TR_U; ++u) add_vec16<DT, R>(w, B[u], emax);
  }
  for (int64_t j = nb * TR_U; j < cnt; ++j) add_vec16<DT, R>(w, ldg_stream(p + j * TR_T), emax);
  if (blockIdx.x == 0 && t < a.head) add_one_elem<DT, R>(w, load_one<DT>(a.x, t), emax);
  if (blockIdx.x == G - 1 && t < a.tail) add_one_elem<DT, R>(w, load_one<DT>(a.x, a.n - a.tail + t), emax);
  w.regularise();
  tops[t] = w.top;

  // special values and signed zeros: exact rescan only when needed
  uint32_t flags = 24u;
  if (emax == Geometry<DT>::EXP_SPECIAL || emax == 0u) {
    flags = 0;
    const char* base = (const char*)a.x + a.head * EB;
    for (int64_t v = vb + t; v < ve; v += TR_T)
      for (int e = 0; e < EPV; ++e) flags |= classify<DT>(load_one<DT>(base, v * EPV + e));
    if (blockIdx.x == 0 && t < a.head) flags |= classify<DT>(load_one<DT>(a.x, t));
    if (blockIdx.x == G - 1 && t < a.tail) flags |= classify<DT>(load_one<DT>(a.x, a.n - a.tail + t));
  }
  __syncthreads();
  if (flags) atomicOr(&blk_flags, flags);
  if (w.events) {
    atomicAdd(&blk_events, w.events);
    atomicMax(&blk_maxdrop, w.low);  // every dropped item lies at a digit <= low
  }

  // ---- CTA merge: the threads' windows, exactly ----
  for (int i = warp; i < ACC_DIGITS; i += NW) {
    int64_t s = 0;
    for (int j = lane; j < TR_T; j += 32) {
      const int sl = i - tops[j] + R - 1;  // slot of digit i in thread j's window
      if (tops[j] >= 0 && sl >= 0 && sl < R) s += tr_cols[sl * TR_T + j];
    }
    s = warp_sum(s);
    if (lane == 0) blk[i] = s;
  }
  __syncthreads();
  if (t < ACC_WORDS - ACC_DIGITS)
    blk[ACC_DIGITS + t] = flag_word(ACC_DIGITS + t, blk_flags, blockIdx.x == 0 ? a.n : 0);
  if (t == 0) {
    if (blk_events) atomicAdd(&a.state[0], blk_events);
    if (blk_maxdrop >= 0) atomicMax(&a.state[1], (unsigned long long)(blk_maxdrop + 1));
  }
  __syncthreads();
  if (t < ACC_WORDS) a.partials[blockIdx.x * ACC_WORDS + t] = blk[t];
  __threadfence();
  __syncthreads();
  if (t == 0) is_last = (atomicAdd(a.ticket, 1u) == (unsigned)(G - 1)) ? 1u : 0u;
  __syncthreads();
  if (!is_last) return;

  // ---- last CTA: merge the partials, round, stopping condition ----
  __threadfence();
  if (t < ACC_WORDS) {
    int64_t s = 0;
    for (int64_t r = 0; r < G; ++r) s += __ldcg((const long long*)a.partials + r * ACC_WORDS + t);
    blk[t] = s;
  }
  __syncthreads();
  if (t == 0) {
    *a.ticket = 0u;
    regularise72(blk);
    const uint64_t y = finalize_acc(blk, limbs, DT, a.out, a.mode);
    const unsigned long long ev = __ldcg(&a.state[0]);
    const int md = (int)__ldcg(&a.state[1]) - 1;
    unsigned long long stop = 1;
    if (ev > 0 && (md < 0 || md + 1 >= ACC_DIGITS)) stop = 0;  // no usable bound: go on
    else if (ev > 0) {
      // B = ev * 2^(32 md + 52) = (ev * 2^20) at digit md + 1
      const int64_t b = (int64_t)(ev << 20);
      for (int sgn = -1; sgn <= 1 && stop; sgn += 2) {
        for (int k = 0; k < ACC_WORDS; ++k) tmp[k] = blk[k];
        tmp[md + 1] += sgn * b;
        regularise72(tmp);
        if (finalize_acc(tmp, limbs, DT, a.out, a.mode) != y) stop = 0;
      }
    }
    store_result(a.result, a.out, y);
    a.state[2] = stop;
  }
}

template <int DT, int R>
static cudaError_t launch_trunc_t(const TruncArgs& a, int max_ctas, cudaStream_t stream) {
  constexpr size_t SMEM = (size_t)R * TR_T * sizeof(int64_t);
  static std::atomic<bool> configured[64] = {};  // idempotent set-up; atomic for concurrent first calls
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !configured[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(trunc_sum_kernel<DT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev].store(true, std::memory_order_release);
  }
  const int64_t want = (a.nvec + 2 * TR_T - 1) / (2 * TR_T);
  const int grid = (int)(want < 1 ? 1 : (want > max_ctas ? max_ctas : want));
  trunc_sum_kernel<DT, R><<<grid, TR_T, SMEM, stream>>>(a);
  return cudaGetLastError();
}

// Load every truncated-pass kernel on the current device now.
cudaError_t trunc_preload() {
  cudaFuncAttributes at;
  const void* fns[] = {(const void*)trunc_sum_kernel<F64, 2>,  (const void*)trunc_sum_kernel<F64, 4>,
                       (const void*)trunc_sum_kernel<F64, 16>, (const void*)trunc_sum_kernel<F32, 2>,
                       (const void*)trunc_sum_kernel<F32, 4>,  (const void*)trunc_sum_kernel<F32, 16>,
                       (const void*)trunc_sum_kernel<BF16, 2>, (const void*)trunc_sum_kernel<BF16, 4>,
                       (const void*)trunc_sum_kernel<BF16, 16>};
  for (const void* f : fns) {
    const cudaError_t e = cudaFuncGetAttributes(&at, f);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int DT>
static cudaError_t launch_trunc_dt(int R, const TruncArgs& a, int max_ctas, cudaStream_t stream) {
  switch (R) {
    case 2: return launch_trunc_t<DT, 2>(a, max_ctas, stream);
    case 4: return launch_trunc_t<DT, 4>(a, max_ctas, stream);
    default: return launch_trunc_t<DT, 16>(a, max_ctas, stream);
  }
}

static cudaError_t launch_trunc(int in_dt, int R, const TruncArgs& a, int max_ctas, cudaStream_t stream) {
  switch (in_dt) {
    case F64: return launch_trunc_dt<F64>(R, a, max_ctas, stream);
    case F32: return launch_trunc_dt<F32>(R, a, max_ctas, stream);
    default: return launch_trunc_dt<BF16>(R, a, max_ctas, stream);
  }
}

}  // namespace es

extern "C" exactsum_status exactsum_sum_adaptive(exactsum_t h, const void* d_x, int64_t n, exactsum_dtype in_dtype,
                                                 exactsum_dtype out_dtype, exactsum_round mode, void* d_result, int* passes,
                                                 int* last_r, exactsum_stream_t stream) {
  exactsum_status st = es_check_common(h, d_x, n, in_dtype, out_dtype, mode, d_result);
  if (st != EXACTSUM_OK) return st;
  if (cudaSetDevice(h->device) != cudaSuccess) return es_cuda_fail(h, cudaGetLastError(), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (!h->trunc_state) {
    if ((e = cudaMalloc(&h->trunc_state, 64)) != cudaSuccess) return es_cuda_fail(h, e, "cudaMalloc(state)");
    if ((e = cudaMallocHost(&h->trunc_state_host, 64)) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaMallocHost(state)");
  }
  // digits a format's exact sum can occupy: above this R nothing is truncated
  const int digits = in_dtype == EXACTSUM_F64 ? 67 : (in_dtype == EXACTSUM_F32 ? 10 : 9);
  const es::SumArgs base = es_make_sum_args(d_x, n, in_dtype);
  int pass = 0;
  for (int R = 2; R < digits && n > 0; R = R * R) {
    ++pass;
    es::TruncArgs a;
    a.x = base.x;
    a.n = base.n;
    a.head = base.head;
    a.nvec = base.nvec;
    a.tail = base.tail;
    a.out = out_dtype;
    a.mode = mode;
    a.result = d_result;
    a.partials = h->partials;
    a.ticket = h->ticket;
    a.state = h->trunc_state;
    if ((e = cudaMemsetAsync(h->trunc_state, 0, 64, s)) != cudaSuccess) return es_cuda_fail(h, e, "cudaMemsetAsync");
    if ((e = es::launch_trunc(in_dtype, R, a, h->max_ctas, s)) != cudaSuccess)
      return es_cuda_fail(h, e, "truncated sum kernel launch");
    if ((e = cudaMemcpyAsync(h->trunc_state_host, h->trunc_state, 64, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return es_cuda_fail(h, e, "cudaMemcpyAsync(state)");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return es_cuda_fail(h, e, "cudaStreamSynchronize");
    if (h->trunc_state_host[2]) {
      if (passes) *passes = pass;
      if (last_r) *last_r = R;
      return EXACTSUM_OK;
    }
  }
  // untruncated: the exact single-pass sum
  st = exactsum_sum(h, d_x, n, in_dtype, out_dtype, mode, d_result, stream);
  if (st != EXACTSUM_OK) return st;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return es_cuda_fail(h, e, "cudaStreamSynchronize");
  if (passes) *passes = pass + 1;
  if (last_r) *last_r = 0;
  return EXACTSUM_OK;
}
