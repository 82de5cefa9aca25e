// sum_bf16.cu -- BF16 single-array exact sums on FP32 digit columns.
//
// The digits are added on the FMA pipe (fdigits.cuh: every element scaled
// into one of 32 FP32 digits by one FFMA, exact for up to 514 additions per
// digit, then flushed into integer digits), so that the integer pipe, which
// bounds the integer-digit form, is left for the address and bit work.
// Two forms: sum_kernel_bf16t, whose input streams through a shared-memory
// ring of bulk asynchronous copies (TMA), and sum_kernel_bf16f, which loads
// it into registers.  Merging and rounding are those of every single-array
// kernel (sum_common.cuh), halving the sum first (the FP32 digits count in
// half units of the BF16 smallest subnormal).
#include <cuda_runtime.h>

#include <atomic>

#include "fdigits.cuh"
#include "sum_common.cuh"
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
// Shapes: sum_kernel_bf16f<ES_BF16F_T, ES_BF16F_U> (register loads) and
// sum_kernel_bf16t<ES_BF16T_C, ES_BF16T_U, ES_BF16T_S> (TMA ring).
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
// Digit stride of the TMA form's columns: the consumer count rounded up to a
// multiple of 256 (ES_BF16T_PAD = 1), so that a digit's byte offset is the
// element's masked exponent bits times a constant (one multiply-add; see
// fdig_add_pair), or the consumer count itself (ES_BF16T_PAD = 0).
#ifndef ES_BF16T_PAD
#define ES_BF16T_PAD 1
#endif
__host__ __device__ constexpr int bf16t_stride(int consumer_warps) {
  return ES_BF16T_PAD ? (consumer_warps * 32 + 255) / 256 * 256 : consumer_warps * 32;
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
  constexpr int FS = bf16t_stride(C);  // digit stride of the columns, in 4-byte words
  constexpr size_t DIG_BYTES = ((size_t)FDIG_INT_DIGITS * FS * 4 + 127) / 128 * 128;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* fd = reinterpret_cast<float*>(smem_raw);                              // 32 (33) x T
  uint4* ring = reinterpret_cast<uint4*>(smem_raw + DIG_BYTES);                // S x BATCH
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)S * BATCH);      // S
  uint64_t* empty = full + S;                                                   // S
  __shared__ int64_t blk[ACC_WORDS];
  __shared__ uint32_t limbs[ACC_DIGITS];
  __shared__ uint32_t blk_flags, is_last;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  pdl_signal();
  const int64_t G = gridDim.x;
  int64_t vb, ve;
  cta_range(a.nvec, vb, ve);
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
  // (columns T .. FS - 1 are padding: they stay zero, also for the CTA merge)
  for (int i = t; i < FDIG_INT_DIGITS * FS; i += NW * 32) fd[i] = 0.0f;
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
    auto flush = [&]() { fdig_flush_warp<FS>(wcols, lane, wd, spec); };
#else
    int32_t I[FDIG_INT_DIGITS];
#pragma unroll
    for (int i = 0; i < FDIG_INT_DIGITS; ++i) I[i] = 0;
    int flushes = 0;
    auto flush = [&]() {
      fdig_flush_regs<FS>(fc, I, spec);
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
        for (int u = 0; u < U; ++u) fdig_add_vec<FS>(fc, r[u]);
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (t + u * T < nv) r[u] = lds128(st + t + u * T);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (t + u * T < nv) fdig_add_vec<FS>(fc, r[u]);
      }
      if (++since_flush == FLUSH_BATCHES) {
        flush();
        since_flush = 0;
      }
    }
    if (!ok && lane == 0) atomicOr(a.status, STATUS_TIMEOUT);
    if (blockIdx.x == 0 && t < a.head) fdig_add_one<FS>(fc, (uint32_t)load_one<BF16>(a.x, t));
    if (blockIdx.x == G - 1 && t < a.tail) fdig_add_one<FS>(fc, (uint32_t)load_one<BF16>(a.x, a.n - a.tail + t));
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
    for (int i = 0; i < FDIG_INT_DIGITS; ++i) ic[i * FS] = I[i];
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
  pdl_wait();
  finish_cta<BF16, C, NW, int64_t, true, (size_t)FDIG_DIGITS * FS * 4>(a, wcol, blk, limbs, blk_flags, &is_last);
#else
  __syncthreads();
  pdl_wait();
  finish_cta<BF16, FS, NW, int32_t, true>(a, reinterpret_cast<int32_t*>(fd), blk, limbs, blk_flags, &is_last);
#endif
}

// launch = false: only load and configure the kernel (see preload_sum_kernels).
static cudaError_t launch_sum_bf16t(const SumArgs& a, int max_ctas, cudaStream_t stream, int* grid_out,
                                    bool launch = true) {
  constexpr int C = ES_BF16T_C, U = ES_BF16T_U, S = ES_BF16T_S;
  constexpr int T = C * 32;
  constexpr size_t DIG_BYTES = ((size_t)FDIG_INT_DIGITS * bf16t_stride(C) * 4 + 127) / 128 * 128;
  constexpr size_t SMEM = DIG_BYTES + (size_t)S * T * U * 16 + 2 * S * 8;
  static_assert(SMEM + 2048 <= 232448, "shared memory per CTA");
  static std::atomic<bool> configured[64] = {};  // idempotent set-up; atomic for concurrent first calls
  cudaError_t e = configure_once((const void*)sum_kernel_bf16t<C, U, S>, SMEM, configured);
  if (e != cudaSuccess || !launch) return e;
  const int64_t want = (a.nvec + 2 * T - 1) / (2 * T);
  const int grid = (int)(want < 1 ? 1 : (want > max_ctas ? max_ctas : want));
  if (grid_out) *grid_out = grid;
  return launch_single_array(sum_kernel_bf16t<C, U, S>, grid, (C + 1) * 32, SMEM, stream, a);
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

cudaError_t launch_sum_bf16(const SumArgs& a, int max_ctas, cudaStream_t stream, int* grid_out, bool launch) {
#if ES_BF16_FFMA == 1
  return launch_sum_bf16f(a, max_ctas, stream, grid_out, launch);
#else
  return launch_sum_bf16t(a, max_ctas, stream, grid_out, launch);
#endif
}

}  // namespace es
