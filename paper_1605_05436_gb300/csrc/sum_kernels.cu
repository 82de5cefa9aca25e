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
// One persistent CTA per SM.  FP64 streams its input through a shared-memory
// ring of bulk asynchronous copies fed by a producer warp (sum_kernel_tma);
// FP32 and BF16 use 16-byte read-only loads, double buffered in registers so
// that each thread keeps two batches in flight (sum_kernel).
#include <cuda_runtime.h>

#include <atomic>

#include "digits.cuh"
#include "fdigits.cuh"
#include "finalize.cuh"
#include "internal.h"
#include "stream.cuh"
#include "tma.cuh"

namespace es {

// BF16 FP32-digit kernel options (measured): batches of L2 prefetch ahead of
// the register loads, and the number of FP32 digit sets per thread (2: the
// two elements of a 32-bit word go to different sets, so their additions
// do not wait on each other).
#ifndef ES_BF16F_PD
#define ES_BF16F_PD 0
#endif
#ifndef ES_BF16F_SETS
#define ES_BF16F_SETS 1
#endif
// BF16 TMA-ring kernel: 1 flushes the FP32 digits warp-transposed into one
// int64 digit per lane (registers freed for more warps); 0 into 33 int32
// digits per thread held in registers.
#ifndef ES_BF16T_WARPFLUSH
#define ES_BF16T_WARPFLUSH 0
#endif

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

// CTA merge and grid merge, shared by both single-array kernels.  Called by
// every thread of the CTA after its flags are in blk_flags and a barrier.
// TC threads own digit columns (digit-major, stride TC); NW warps take part.
// HALF: the columns count in half units of the input format (the BF16
// FP32-digit columns, fdigits.cuh); their exact sum is even and is halved
// here, digit by digit, before it leaves the CTA.
// SCRATCH: bytes available at `cols` (reused for the grid merge).
template <int DT, int TC, int NW, typename D, bool HALF = false,
          size_t SCRATCH = (size_t)Geometry<DT>::DIGITS * TC * sizeof(D)>
__device__ __forceinline__ void finish_cta(const SumArgs& a, D* cols, int64_t* blk, uint32_t* limbs,
                                           uint32_t blk_flags, uint32_t* is_last) {
  static_assert(SCRATCH >= NW * ACC_WORDS * sizeof(int64_t), "digit area reused for the grid merge");
  int64_t* digits = reinterpret_cast<int64_t*>(cols);  // scratch once the columns are merged
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t G = gridDim.x;
  // ---- CTA merge: sum the columns' digits, carry-free ----
  for (int i = warp; i < ACC_DIGITS; i += NW) {
    int64_t s = 0;
    for (int j = lane; j < TC; j += 32) s += digit32<DT, TC>(cols + j, i);
    s = warp_sum(s);
    if (lane == 0) blk[i] = s;
  }
  if (t < ACC_WORDS - ACC_DIGITS)
    blk[ACC_DIGITS + t] = flag_word(ACC_DIGITS + t, blk_flags, blockIdx.x == 0 ? a.n : 0);
  __syncthreads();
  if constexpr (HALF) {
    // V = sum D_i 2^(32 i) is even, so D_0 is even and
    // V / 2 = sum ((D_i >> 1) + (D_(i+1) & 1) 2^31) 2^(32 i)
    int64_t v = 0, up = 0;
    if (t < ACC_DIGITS) {
      v = blk[t];
      up = (t + 1 < ACC_DIGITS) ? blk[t + 1] : 0;
    }
    __syncthreads();
    if (t < ACC_DIGITS) blk[t] = (v >> 1) + ((up & 1) << 31);
    __syncthreads();
  }
  if (t < ACC_WORDS) a.partials[blockIdx.x * ACC_WORDS + t] = blk[t];
  __threadfence();
  __syncthreads();
  if (t == 0) *is_last = (atomicAdd(a.ticket, 1u) == (unsigned)(G - 1)) ? 1u : 0u;
  __syncthreads();
  if (!*is_last) return;

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

// Register-streaming form: every thread loads its own vectors (16-byte
// read-only loads, double buffered) and owns one digit column of type D
// (int64, or int32 for BF16).
template <int DT, int T, int U, typename D>
__global__ void __launch_bounds__(T, 1) sum_kernel(SumArgs a) {
  constexpr int ND = ColumnDigits<DT, D>::value;
  constexpr int REG_EVERY = RegEvery<DT, D>::value;
  constexpr int NW = T / 32;

  extern __shared__ int64_t smem_digits[];  // ND x T digits of type D
  D* digits = reinterpret_cast<D*>(smem_digits);
  __shared__ int64_t blk[ACC_WORDS];
  __shared__ uint32_t limbs[ACC_DIGITS];
  __shared__ uint32_t blk_flags, is_last;

  const int t = threadIdx.x;
  D* col = digits + t;
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
  emax = emax_unpack<DT, D>(emax);

  // ---- unaligned head (CTA 0) and ragged tail (last CTA) ----
  if (blockIdx.x == 0 && t < a.head) add_one<DT, T>(col, load_one<DT>(a.x, t), emax);
  if (blockIdx.x == G - 1 && t < a.tail) add_one<DT, T>(col, load_one<DT>(a.x, a.n - a.tail + t), emax);
  regularise<DT, T>(col);

  // ---- special values and signed zeros: exact rescan only when needed ----
  uint32_t flags = 24u;  // an element with 0 < E < all-ones is neither +0 nor -0
  if (emax == Geometry<DT>::EXP_SPECIAL || emax == 0u) flags = rescan_flags<DT, T>(a, vb, ve);
  __syncthreads();
  if (flags) atomicOr(&blk_flags, flags);
  __syncthreads();
  finish_cta<DT, T, NW, D>(a, digits, blk, limbs, blk_flags, &is_last);
}

// BF16 with FP32 digit columns (fdigits.cuh): every thread owns 32 FP32
// digits, added by one FFMA per element, and 33 int32 digits that take the
// FP32 digits at each flush (at most FDIG_MAX_ADDS additions per FP32 digit
// in between).  16-byte read-only loads, double buffered as in sum_kernel.
// Specials are caught by the flushes (a digit became non-finite); a thread
// whose digits end all zero saw only zeros or a sum that cancelled, and
// rescans its elements for the signed-zero flags.
template <int T, int U>
__global__ void __launch_bounds__(T, 1) sum_kernel_bf16f(SumArgs a) {
  constexpr int NW = T / 32;
  constexpr int EPB = U * 8;  // elements per batch
  // flush before a batch could take a digit past FDIG_MAX_ADDS additions,
  // counting the U - 1 leftover vectors and the head and tail element
  constexpr int FLUSH_BATCHES = (FDIG_MAX_ADDS - 2 - (U - 1) * 8) / EPB;
  static_assert(FLUSH_BATCHES >= 1, "batch too large for the FP32 digits");

  constexpr int SETS = ES_BF16F_SETS;
  extern __shared__ int64_t smem_digits[];
  float* fd = reinterpret_cast<float*>(smem_digits);                     // SETS x 32 x T
  int32_t* id = reinterpret_cast<int32_t*>(fd + SETS * FDIG_DIGITS * T); // 33 x T
  __shared__ int64_t blk[ACC_WORDS];
  __shared__ uint32_t limbs[ACC_DIGITS];
  __shared__ uint32_t blk_flags, is_last;

  const int t = threadIdx.x;
  float* fc = fd + t;
  float* fc1 = fd + (SETS - 1) * FDIG_DIGITS * T + t;
  int32_t* ic = id + t;
#pragma unroll 4
  for (int i = 0; i < SETS * FDIG_DIGITS; ++i) fc[i * T] = 0.0f;
#pragma unroll 4
  for (int i = 0; i < FDIG_INT_DIGITS; ++i) ic[i * T] = 0;
  if (t == 0) blk_flags = 0;

  const uint4* vx = reinterpret_cast<const uint4*>((const char*)a.x + a.head * 2);
  const int64_t G = gridDim.x;
  const int64_t vb = a.nvec * blockIdx.x / G, ve = a.nvec * (blockIdx.x + 1) / G;
  const int64_t cnt = (vb + t < ve) ? (ve - vb - t + T - 1) / T : 0;
  const uint4* p = vx + vb + t;
  constexpr int64_t PER = (int64_t)T * U;
  const int64_t nb = cnt / U;
  uint32_t spec = 0;
  int since_flush = 0, flushes = 0;
  auto flush = [&]() {
    fdig_flush<T>(fc, ic, spec);
    if constexpr (SETS == 2) fdig_flush<T>(fc1, ic, spec);
  };
  auto add_vec = [&](const uint4& v) {
    if constexpr (SETS == 2) fdig_add_vec2<T>(fc, fc1, v);
    else fdig_add_vec<T>(fc, v);
  };
  auto after_batch = [&]() {
    if (++since_flush == FLUSH_BATCHES) {
      flush();
      since_flush = 0;
      if (++flushes == FDIG_REG_FLUSHES / SETS) {
        fdig_regularise<T>(ic);
        flushes = 0;
      }
    }
  };

  // ---- hot loop: this thread's vectors vb + t + j*T, double buffered ----
  // (ES_BF16F_PD > 0: thread 0 also asks for the CTA's batch PD ahead to be
  // brought into L2, so that the register loads find it there)
  constexpr int PD = ES_BF16F_PD;
  const uint4* cta_end = vx + ve;
  auto prefetch = [&](int64_t kb) {
    const uint4* q = vx + vb + kb * PER;
    if (q < cta_end) prefetch_l2(q, (uint32_t)(min(PER, (int64_t)(cta_end - q)) * 16));
  };
  if (PD > 0 && t == 0)
    for (int k = 0; k < PD; ++k) prefetch(k);
  uint4 A[U], B[U];
  if (nb > 0) {
#pragma unroll
    for (int u = 0; u < U; ++u) A[u] = ldg_stream(p + u * T);
  }
  for (int64_t k = 0; k < nb; k += 2) {
    if (PD > 0 && t == 0) {
      prefetch(k + PD);
      prefetch(k + PD + 1);
    }
    if (k + 1 < nb) {
#pragma unroll
      for (int u = 0; u < U; ++u) B[u] = ldg_stream(p + (k + 1) * PER + u * T);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) add_vec(A[u]);
    after_batch();
    if (k + 1 >= nb) break;
    if (k + 2 < nb) {
#pragma unroll
      for (int u = 0; u < U; ++u) A[u] = ldg_stream(p + (k + 2) * PER + u * T);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) add_vec(B[u]);
    after_batch();
  }
  for (int64_t j = nb * U; j < cnt; ++j) add_vec(ldg_stream(p + j * T));

  // ---- unaligned head (CTA 0) and ragged tail (last CTA) ----
  if (blockIdx.x == 0 && t < a.head) fdig_add_one<T>(fc, (uint32_t)load_one<BF16>(a.x, t));
  if (blockIdx.x == G - 1 && t < a.tail) fdig_add_one<T>(fc, (uint32_t)load_one<BF16>(a.x, a.n - a.tail + t));
  flush();
  fdig_regularise<T>(ic);

  // ---- special values and signed zeros: exact rescan only when needed ----
  uint32_t any = 0;
#pragma unroll 4
  for (int i = 0; i < FDIG_INT_DIGITS; ++i) any |= (uint32_t)ic[i * T];
  uint32_t flags = 24u;  // a thread with a non-zero digit saw a non-zero element
  if (spec == 0x7F800000u || any == 0u) flags = rescan_flags<BF16, T>(a, vb, ve);
  __syncthreads();
  if (flags) atomicOr(&blk_flags, flags);
  __syncthreads();
  finish_cta<BF16, T, NW, int32_t, true>(a, id, blk, limbs, blk_flags, &is_last);
}

// BF16 with FP32 digit columns fed by a TMA ring: one producer warp streams
// the CTA's range through S shared-memory stages of C*32*U vectors with bulk
// asynchronous copies (as sum_kernel_tma does for FP64); C consumer warps
// read their U vectors of a stage, release it and add the elements into
// their FP32 digits (fdigits.cuh).  The int32 digits that the FP32 digits
// are flushed into live in registers (33 per thread), so a flush costs two
// shared-memory accesses per digit.
template <int C, int U, int S>
__global__ void __launch_bounds__((C + 1) * 32, 1) sum_kernel_bf16t(SumArgs a) {
  constexpr int T = C * 32;          // consumer threads (digit columns)
  constexpr int NW = C + 1;
  constexpr int BATCH = T * U;       // vectors per stage
  constexpr int EPB = U * 8;         // elements per consumer thread per stage
  constexpr int FLUSH_BATCHES = (FDIG_MAX_ADDS - 2) / EPB;
  static_assert(FLUSH_BATCHES >= 1, "stage too large for the FP32 digits");
  constexpr size_t DIG_BYTES = ((size_t)FDIG_INT_DIGITS * T * 4 + 127) / 128 * 128;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* fd = reinterpret_cast<float*>(smem_raw);                              // 32 (33) x T
  uint4* ring = reinterpret_cast<uint4*>(smem_raw + DIG_BYTES);                // S x BATCH
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)S * BATCH);      // S
  uint64_t* empty = full + S;                                                   // S
  __shared__ int64_t blk[ACC_WORDS];
  __shared__ uint32_t limbs[ACC_DIGITS];
  __shared__ uint32_t blk_flags, is_last;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t G = gridDim.x;
  const int64_t vb = a.nvec * blockIdx.x / G, ve = a.nvec * (blockIdx.x + 1) / G;
  const int64_t nv_cta = ve - vb;
  const int64_t nbatch = (nv_cta + BATCH - 1) / BATCH;
  const uint4* vx = reinterpret_cast<const uint4*>((const char*)a.x + a.head * 2);

  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C);
    }
    blk_flags = 0;
    mbar_init_fence();
  }
  for (int i = t; i < FDIG_DIGITS * T; i += NW * 32) fd[i] = 0.0f;
  __syncthreads();

  uint32_t flags = 0;
  int64_t warp_digit = 0;
  if (warp == C) {
    // ---- producer: one elected lane issues the bulk copies ----
    if (lane == 0) {
      bool ok = true;
      int64_t issued = 0;
      for (int64_t k = 0; k < nbatch; ++k) {
        const int s = (int)(k % S);
        if (k >= S && !mbar_wait(&empty[s], (uint32_t)((k / S - 1) & 1))) {
          ok = false;
          break;
        }
        const int64_t nv = min((int64_t)BATCH, nv_cta - k * BATCH);
        mbar_arrive_expect_tx(&full[s], (uint32_t)(nv * 16));
        bulk_copy_g2s(ring + (size_t)s * BATCH, vx + vb + k * BATCH, (uint32_t)(nv * 16), &full[s]);
        issued = k + 1;
      }
      // never leave copies in flight: wait (bounded) for the last ones to land
      for (int64_t k = (issued > S ? issued - S : 0); k < issued; ++k)
        ok &= mbar_wait(&full[k % S], (uint32_t)((k / S) & 1));
      if (!ok) atomicOr(a.status, STATUS_TIMEOUT);
    }
  } else {
    // ---- consumers ----
    float* fc = fd + t;
    uint32_t spec = 0;
#if ES_BF16T_WARPFLUSH
    int64_t wd = 0;  // digit `lane` of this warp's int64 accumulator
    float* wcols = fd + warp * 32;
    auto flush = [&]() { fdig_flush_warp<T>(wcols, lane, wd, spec); };
#else
    int32_t I[FDIG_INT_DIGITS];
#pragma unroll
    for (int i = 0; i < FDIG_INT_DIGITS; ++i) I[i] = 0;
    int flushes = 0;
    auto flush = [&]() {
      fdig_flush_regs<T>(fc, I, spec);
      if (++flushes == FDIG_REG_FLUSHES) {
        fdig_regularise_regs(I);
        flushes = 0;
      }
    };
#endif
    int since_flush = 0;
    bool ok = true;
    for (int64_t k = 0; k < nbatch; ++k) {
      const int s = (int)(k % S);
      // a lane whose bounded wait gave up stays in the loop (without waiting
      // again, its result already invalid) so that every lane of the warp
      // meets the same warp barriers and flushes
      if (ok && !mbar_wait(&full[s], (uint32_t)((k / S) & 1))) ok = false;
      const int64_t nv = min((int64_t)BATCH, nv_cta - k * BATCH);
      const uint4* st = ring + (size_t)s * BATCH;
      uint4 r[U];
      if (nv == BATCH) {
#pragma unroll
        for (int u = 0; u < U; ++u) r[u] = lds128(st + t + u * T);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
        for (int u = 0; u < U; ++u) fdig_add_vec<T>(fc, r[u]);
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (t + u * T < nv) r[u] = lds128(st + t + u * T);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (t + u * T < nv) fdig_add_vec<T>(fc, r[u]);
      }
      if (++since_flush == FLUSH_BATCHES) {
        flush();
        since_flush = 0;
      }
    }
    if (!ok && lane == 0) atomicOr(a.status, STATUS_TIMEOUT);
    if (blockIdx.x == 0 && t < a.head) fdig_add_one<T>(fc, (uint32_t)load_one<BF16>(a.x, t));
    if (blockIdx.x == G - 1 && t < a.tail) fdig_add_one<T>(fc, (uint32_t)load_one<BF16>(a.x, a.n - a.tail + t));
    flush();
#if ES_BF16T_WARPFLUSH
    // specials and all-zero digits are judged per warp (the flags only
    // matter OR-ed over the CTA): a warp whose digits are not all zero saw a
    // non-zero element
    const bool warp_special = __any_sync(0xffffffffu, spec == 0x7F800000u);
    const bool warp_zero = !__any_sync(0xffffffffu, wd != 0);
    flags = 24u;
    if (warp_special || warp_zero) flags = rescan_flags<BF16, T>(a, vb, ve);
#else
    fdig_regularise_regs(I);
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < FDIG_INT_DIGITS; ++i) any |= (uint32_t)I[i];
    // consumer thread t owns vectors vb + t + j*T: the same sets as the
    // register-streaming form, so the same exact rescan applies
    flags = 24u;
    if (spec == 0x7F800000u || any == 0u) flags = rescan_flags<BF16, T>(a, vb, ve);
    // the int32 digits take the place of the FP32 digits for the CTA merge
    int32_t* ic = reinterpret_cast<int32_t*>(fd) + t;
#pragma unroll
    for (int i = 0; i < FDIG_INT_DIGITS; ++i) ic[i * T] = I[i];
#endif
#if ES_BF16T_WARPFLUSH
    warp_digit = wd;
#endif
  }
  __syncthreads();
  if (flags) atomicOr(&blk_flags, flags);
#if ES_BF16T_WARPFLUSH
  // one int64 column of 33 radix-2^8 digits per consumer warp (digit 32,
  // the carry digit, stays zero), in the FP32 digit area
  int64_t* wcol = reinterpret_cast<int64_t*>(fd);
  if (warp < C) {
    wcol[lane * C + warp] = warp_digit;
    if (lane == 0) wcol[32 * C + warp] = 0;
  }
  __syncthreads();
  finish_cta<BF16, C, NW, int64_t, true, (size_t)FDIG_DIGITS * T * 4>(a, wcol, blk, limbs, blk_flags, &is_last);
#else
  __syncthreads();
  finish_cta<BF16, T, NW, int32_t, true>(a, reinterpret_cast<int32_t*>(fd), blk, limbs, blk_flags, &is_last);
#endif
}

// TMA-streaming form: one producer warp moves the CTA's range through a ring
// of S shared-memory stages with bulk asynchronous copies (cp.async.bulk,
// completion tracked by mbarriers); C consumer warps read their vectors from
// the ring, release the stage at once and add the elements into their
// digit columns.  The bytes in flight live in shared memory rather than in
// registers, so a CTA keeps S stages of the input in flight.
template <int DT, int C, int U, int S>
__global__ void __launch_bounds__((C + 1) * 32, 1) sum_kernel_tma(SumArgs a) {
  constexpr int T = C * 32;          // consumer threads (digit columns)
  constexpr int NW = C + 1;
  constexpr int ND = Geometry<DT>::DIGITS;
  constexpr int REG_EVERY = Geometry<DT>::REG_EVERY;
  constexpr int EPV = 16 / Geometry<DT>::ELEM_BYTES;
  constexpr int BATCH = T * U;       // vectors per stage

  extern __shared__ __align__(128) unsigned char smem_raw[];
  int64_t* digits = reinterpret_cast<int64_t*>(smem_raw);                       // ND x T
  uint4* ring = reinterpret_cast<uint4*>(smem_raw + (size_t)ND * T * 8);        // S x BATCH
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)S * BATCH);       // S
  uint64_t* empty = full + S;                                                    // S
  __shared__ int64_t blk[ACC_WORDS];
  __shared__ uint32_t limbs[ACC_DIGITS];
  __shared__ uint32_t blk_flags, is_last;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t G = gridDim.x;
  const int64_t vb = a.nvec * blockIdx.x / G, ve = a.nvec * (blockIdx.x + 1) / G;
  const int64_t nv_cta = ve - vb;
  const int64_t nbatch = (nv_cta + BATCH - 1) / BATCH;
  const uint4* vx = reinterpret_cast<const uint4*>((const char*)a.x + a.head * Geometry<DT>::ELEM_BYTES);

  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C);
    }
    blk_flags = 0;
    mbar_init_fence();
  }
  __syncthreads();

  uint32_t flags = 0;
  if (warp == C) {
    // ---- producer: one elected lane issues the bulk copies ----
    if (lane == 0) {
      bool ok = true;
      int64_t issued = 0;
      for (int64_t k = 0; k < nbatch; ++k) {
        const int s = (int)(k % S);
        if (k >= S && !mbar_wait(&empty[s], (uint32_t)((k / S - 1) & 1))) {
          ok = false;
          break;
        }
        const int64_t nv = min((int64_t)BATCH, nv_cta - k * BATCH);
        mbar_arrive_expect_tx(&full[s], (uint32_t)(nv * 16));
        bulk_copy_g2s(ring + (size_t)s * BATCH, vx + vb + k * BATCH, (uint32_t)(nv * 16), &full[s]);
        issued = k + 1;
      }
      // never leave copies in flight: wait (bounded) for the last ones to land
      for (int64_t k = (issued > S ? issued - S : 0); k < issued; ++k)
        ok &= mbar_wait(&full[k % S], (uint32_t)((k / S) & 1));
      if (!ok) atomicOr(a.status, STATUS_TIMEOUT);
    }
  } else {
    // ---- consumers ----
    int64_t* col = digits + t;
#pragma unroll 4
    for (int i = 0; i < ND; ++i) col[i * T] = 0;
    uint32_t emax = 0;
    int reg_left = REG_EVERY;
    bool ok = true;
    for (int64_t k = 0; k < nbatch; ++k) {
      const int s = (int)(k % S);
      if (!mbar_wait(&full[s], (uint32_t)((k / S) & 1))) {
        ok = false;
        break;
      }
      const int64_t nv = min((int64_t)BATCH, nv_cta - k * BATCH);
      const uint4* st = ring + (size_t)s * BATCH;
      uint4 r[U];
      if (nv == BATCH) {
#pragma unroll
        for (int u = 0; u < U; ++u) r[u] = lds128(st + t + u * T);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
        for (int u = 0; u < U; ++u) add_vec<DT, T>(col, r[u], emax);
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (t + u * T < nv) r[u] = lds128(st + t + u * T);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (t + u * T < nv) add_vec<DT, T>(col, r[u], emax);
      }
      reg_left -= U * EPV;
      if (reg_left <= 0) {
        regularise<DT, T>(col);
        reg_left = REG_EVERY;
      }
    }
    if (!ok && lane == 0) atomicOr(a.status, STATUS_TIMEOUT);
    if (blockIdx.x == 0 && t < a.head) add_one<DT, T>(col, load_one<DT>(a.x, t), emax);
    if (blockIdx.x == G - 1 && t < a.tail) add_one<DT, T>(col, load_one<DT>(a.x, a.n - a.tail + t), emax);
    regularise<DT, T>(col);
    // consumer thread t owns vectors vb + t + j*T: the same sets as the
    // register-streaming form, so the same exact rescan applies
    flags = 24u;
    if (emax == Geometry<DT>::EXP_SPECIAL || emax == 0u) flags = rescan_flags<DT, T>(a, vb, ve);
  }
  __syncthreads();
  if (flags) atomicOr(&blk_flags, flags);
  __syncthreads();
  finish_cta<DT, T, NW, int64_t>(a, digits, blk, limbs, blk_flags, &is_last);
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
// Streaming form and shape per input format (chosen by measurement):
//   TMA = 1: sum_kernel_tma<DT, C, TU, S>, (C + 1) warps, S stages of C*32*TU vectors;
//   TMA = 0: sum_kernel<DT, T, U>, T threads, U vectors per batch.
// Digit columns: int64 for FP64; for FP32 radix-2^16 sign-split unsigned
// 64-bit halves (ES_F32_R16 = 1; else radix-2^8 int64); for BF16 sign-split
// unsigned 32-bit halves (ES_BF16_SPLIT = 1), else signed int32
// (ES_BF16_I32 = 1) or int64.
#ifndef ES_F64_TMA
#define ES_F64_TMA 1
#endif
#ifndef ES_F64_C
#define ES_F64_C 8
#endif
#ifndef ES_F64_TU
#define ES_F64_TU 10
#endif
#ifndef ES_F64_S
#define ES_F64_S 2
#endif
#ifndef ES_F64_T
#define ES_F64_T 384
#endif
#ifndef ES_F64_U
#define ES_F64_U 8
#endif
#ifndef ES_F32_TMA
#define ES_F32_TMA 0
#endif
#ifndef ES_F32_C
#define ES_F32_C 12
#endif
#ifndef ES_F32_TU
#define ES_F32_TU 4
#endif
#ifndef ES_F32_S
#define ES_F32_S 4
#endif
#ifndef ES_F32_T
#define ES_F32_T 640
#endif
#ifndef ES_F32_U
#define ES_F32_U 5
#endif
#ifndef ES_BF16_TMA
#define ES_BF16_TMA 0
#endif
#ifndef ES_BF16_C
#define ES_BF16_C 12
#endif
#ifndef ES_BF16_TU
#define ES_BF16_TU 4
#endif
#ifndef ES_BF16_S
#define ES_BF16_S 4
#endif
#ifndef ES_BF16_T
#define ES_BF16_T 768
#endif
#ifndef ES_BF16_U
#define ES_BF16_U 4
#endif
#ifndef ES_BF16_I32
#define ES_BF16_I32 1
#endif
#ifndef ES_BF16_SPLIT
#define ES_BF16_SPLIT 1
#endif
// BF16 with FP32 digit columns added on the FMA pipe (fdigits.cuh):
// 1: sum_kernel_bf16f<ES_BF16F_T, ES_BF16F_U> (register loads);
// 2: sum_kernel_bf16t<ES_BF16T_C, ES_BF16T_U, ES_BF16T_S> (TMA ring);
// 0 selects the integer columns above.
#ifndef ES_BF16_FFMA
#define ES_BF16_FFMA 2
#endif
#ifndef ES_BF16F_T
#define ES_BF16F_T 768
#endif
#ifndef ES_BF16F_U
#define ES_BF16F_U 4
#endif
#ifndef ES_BF16T_C
#define ES_BF16T_C 27
#endif
#ifndef ES_BF16T_U
#define ES_BF16T_U 3
#endif
#ifndef ES_BF16T_S
#define ES_BF16T_S 2
#endif
template <> struct SumConfig<F64> {
  static constexpr int TMA = ES_F64_TMA, C = ES_F64_C, TU = ES_F64_TU, S = ES_F64_S, T = ES_F64_T, U = ES_F64_U;
  using Digit = int64_t;
};
#ifndef ES_F32_R16
#define ES_F32_R16 1
#endif
template <> struct SumConfig<F32> {
  static constexpr int TMA = ES_F32_TMA, C = ES_F32_C, TU = ES_F32_TU, S = ES_F32_S, T = ES_F32_T, U = ES_F32_U;
#if ES_F32_R16
  using Digit = uint64_t;
#else
  using Digit = int64_t;
#endif
};
template <> struct SumConfig<BF16> {
  static constexpr int TMA = ES_BF16_TMA, C = ES_BF16_C, TU = ES_BF16_TU, S = ES_BF16_S, T = ES_BF16_T,
                       U = ES_BF16_U;
#if ES_BF16_SPLIT
  using Digit = uint32_t;
#elif ES_BF16_I32
  using Digit = int32_t;
#else
  using Digit = int64_t;
#endif
};

// Set the dynamic shared-memory limit of a kernel once per device.
static cudaError_t configure_once(const void* fn, size_t smem, std::atomic<bool>* done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64) done[dev].store(true, std::memory_order_release);
  return cudaSuccess;
}

// launch = false: only load and configure the kernel (see preload_sum_kernels).
static cudaError_t launch_sum_bf16t(const SumArgs& a, int max_ctas, cudaStream_t stream, int* grid_out,
                                    bool launch = true) {
  constexpr int C = ES_BF16T_C, U = ES_BF16T_U, S = ES_BF16T_S;
  constexpr int T = C * 32;
  constexpr size_t DIG_BYTES = ((size_t)FDIG_INT_DIGITS * T * 4 + 127) / 128 * 128;
  constexpr size_t SMEM = DIG_BYTES + (size_t)S * T * U * 16 + 2 * S * 8;
  static_assert(SMEM + 2048 <= 232448, "shared memory per CTA");
  static std::atomic<bool> configured[64] = {};  // idempotent set-up; atomic for concurrent first calls
  cudaError_t e = configure_once((const void*)sum_kernel_bf16t<C, U, S>, SMEM, configured);
  if (e != cudaSuccess || !launch) return e;
  const int64_t want = (a.nvec + 2 * T - 1) / (2 * T);
  const int grid = (int)(want < 1 ? 1 : (want > max_ctas ? max_ctas : want));
  if (grid_out) *grid_out = grid;
  sum_kernel_bf16t<C, U, S><<<grid, (C + 1) * 32, SMEM, stream>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_sum_bf16f(const SumArgs& a, int max_ctas, cudaStream_t stream, int* grid_out,
                                    bool launch = true) {
  constexpr int T = ES_BF16F_T, U = ES_BF16F_U;
  constexpr size_t SMEM = (size_t)(ES_BF16F_SETS * FDIG_DIGITS + FDIG_INT_DIGITS) * T * 4;
  static_assert(SMEM + 2048 <= 232448, "shared memory per CTA");
  static std::atomic<bool> configured[64] = {};  // idempotent set-up; atomic for concurrent first calls
  cudaError_t e = configure_once((const void*)sum_kernel_bf16f<T, U>, SMEM, configured);
  if (e != cudaSuccess || !launch) return e;
  const int64_t want = (a.nvec + 2 * T - 1) / (2 * T);
  const int grid = (int)(want < 1 ? 1 : (want > max_ctas ? max_ctas : want));
  if (grid_out) *grid_out = grid;
  sum_kernel_bf16f<T, U><<<grid, T, SMEM, stream>>>(a);
  return cudaGetLastError();
}

template <int DT>
static cudaError_t launch_sum_t(const SumArgs& a, int max_ctas, cudaStream_t stream, int* grid_out,
                                bool launch = true) {
  if constexpr (DT == BF16 && ES_BF16_FFMA == 2) return launch_sum_bf16t(a, max_ctas, stream, grid_out, launch);
  if constexpr (DT == BF16 && ES_BF16_FFMA == 1) return launch_sum_bf16f(a, max_ctas, stream, grid_out, launch);
  using Cfg = SumConfig<DT>;
  using D = typename Cfg::Digit;
  constexpr int ND = ColumnDigits<DT, D>::value;
  constexpr int THREADS = Cfg::TMA ? (Cfg::C + 1) * 32 : Cfg::T;
  constexpr int COLS = Cfg::TMA ? Cfg::C * 32 : Cfg::T;
  static_assert(!Cfg::TMA || sizeof(D) == 8, "the TMA form keeps int64 digit columns");
  constexpr size_t SMEM = Cfg::TMA ? (size_t)ND * COLS * 8 + (size_t)Cfg::S * COLS * Cfg::TU * 16 + 2 * Cfg::S * 8
                                   : (size_t)ND * COLS * sizeof(D);
  static_assert(!Cfg::TMA || ((size_t)ND * COLS * 8) % 128 == 0, "ring must start 128-byte aligned");
  static_assert(SMEM + 1024 <= 232448, "shared memory per CTA");
  const void* fn;
  if constexpr (Cfg::TMA) fn = (const void*)sum_kernel_tma<DT, Cfg::C, Cfg::TU, Cfg::S>;
  else fn = (const void*)sum_kernel<DT, Cfg::T, Cfg::U, D>;
  static std::atomic<bool> configured[64] = {};  // idempotent set-up; atomic for concurrent first calls
  cudaError_t e = configure_once(fn, SMEM, configured);
  if (e != cudaSuccess || !launch) return e;
  // at least two vectors per column per CTA, at most one CTA per SM
  const int64_t want = (a.nvec + 2 * COLS - 1) / (2 * COLS);
  const int grid = (int)(want < 1 ? 1 : (want > max_ctas ? max_ctas : want));
  if (grid_out) *grid_out = grid;
  if constexpr (Cfg::TMA)
    sum_kernel_tma<DT, Cfg::C, Cfg::TU, Cfg::S><<<grid, THREADS, SMEM, stream>>>(a);
  else
    sum_kernel<DT, Cfg::T, Cfg::U, D><<<grid, THREADS, SMEM, stream>>>(a);
  return cudaGetLastError();
}

// Load and configure the single-array kernels of every input format now
// (setting a kernel's attribute loads a lazily loaded kernel): a first
// launch that has to load its module waits for the kernels already running,
// which a caller with a resident kernel on the device must not meet
// mid-stream.
cudaError_t preload_sum_kernels() {
  const SumArgs none{};
  cudaError_t e = launch_sum_t<F64>(none, 1, nullptr, nullptr, false);
  if (e == cudaSuccess) e = launch_sum_t<F32>(none, 1, nullptr, nullptr, false);
  if (e == cudaSuccess) e = launch_sum_t<BF16>(none, 1, nullptr, nullptr, false);
  cudaFuncAttributes at;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&at, (const void*)round_acc_kernel);
  return e;
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


}  // namespace es
