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
// FP32 uses 16-byte read-only loads, double buffered in registers so that
// each thread keeps two batches in flight (sum_kernel).  BF16 has its own
// kernels on FP32 digit columns (sum_bf16.cu); the integer-column form here
// remains selectable.  The rescan and the CTA and grid merges are in
// sum_common.cuh.
#include <cuda_runtime.h>

#include <atomic>

#include "sum_common.cuh"
#include "tma.cuh"
namespace es {

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
  pdl_signal();
  D* col = digits + t;
#pragma unroll 4
  for (int i = 0; i < ND; ++i) col[i * T] = 0;
  if (t == 0) blk_flags = 0;

  uint32_t emax = 0;
  const uint4* vx = reinterpret_cast<const uint4*>((const char*)a.x + a.head * Geometry<DT>::ELEM_BYTES);
  const int64_t G = gridDim.x;
  int64_t vb, ve;
  cta_range(a.nvec, vb, ve);
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
  pdl_wait();
  finish_cta<DT, T, NW, D>(a, digits, blk, limbs, blk_flags, &is_last);
}

// TMA-streaming form: one producer warp moves the CTA's range through a ring
// of S shared-memory stages with bulk asynchronous copies (cp.async.bulk,
// completion tracked by mbarriers); C consumer warps read their vectors from
// the ring, release the stage at once and add the elements into their
// digit columns.  The bytes in flight live in shared memory rather than in
// registers, so a CTA keeps S stages of the input in flight.
// D: the digit type of the columns (int64 for FP64; the FP32 radix-2^32
// sign-split uint64 columns), 8 bytes either way.
template <int DT, int C, int U, int S, typename D = int64_t>
__global__ void __launch_bounds__((C + 1) * 32, 1) sum_kernel_tma(SumArgs a) {
  static_assert(sizeof(D) == 8, "8-byte digits");
  constexpr int T = C * 32;          // consumer threads (digit columns)
  constexpr int NW = C + 1;
  constexpr int ND = ColumnDigits<DT, D>::value;
  constexpr int REG_EVERY = RegEvery<DT, D>::value;
  constexpr int EPV = 16 / Geometry<DT>::ELEM_BYTES;
  constexpr int BATCH = T * U;       // vectors per stage

  extern __shared__ __align__(128) unsigned char smem_raw[];
  D* digits = reinterpret_cast<D*>(smem_raw);                                    // ND x T
  uint4* ring = reinterpret_cast<uint4*>(smem_raw + (size_t)ND * T * 8);        // S x BATCH
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)S * BATCH);       // S
  uint64_t* empty = full + S;                                                    // S
  __shared__ int64_t blk[ACC_WORDS];
  __shared__ uint32_t limbs[ACC_DIGITS];
  __shared__ uint32_t blk_flags, is_last;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t G = gridDim.x;
#if ES_TAIL_CUT > 0
  // the last CTA takes ES_TAIL_CUT fewer vectors (at most a quarter of a
  // share), the others share them
  const int64_t cut = min((int64_t)ES_TAIL_CUT, a.nvec / (4 * G));
  const int64_t vb = (a.nvec + cut) * blockIdx.x / G;
  const int64_t ve = blockIdx.x == G - 1 ? a.nvec : (a.nvec + cut) * (blockIdx.x + 1) / G;
#else
  const int64_t vb = a.nvec * blockIdx.x / G, ve = a.nvec * (blockIdx.x + 1) / G;
#endif
  const int64_t nv_cta = ve - vb;
  const int64_t nbatch = (nv_cta + BATCH - 1) / BATCH;
  const uint4* vx = reinterpret_cast<const uint4*>((const char*)a.x + a.head * Geometry<DT>::ELEM_BYTES);

#if ES_PDL
  // the next launch on the stream may start its CTAs as this one's leave
  asm volatile("griddepcontrol.launch_dependents;");
#endif
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
    D* col = digits + t;
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
    emax = emax_unpack<DT, D>(emax);
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
#if ES_PDL
  // partials, ticket and result of the launch before are shared: wait for it
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
  finish_cta<DT, T, NW, D>(a, digits, blk, limbs, blk_flags, &is_last);
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
// Digit columns: int64 for FP64; for FP32 sign-split unsigned 64-bit halves
// (ES_F32_R16 = 1: radix 2^32 with ES_F32_R32 = 1, else radix 2^16;
// ES_F32_R16 = 0: radix-2^8 int64); for BF16 sign-split
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
#define ES_F32_T 896
#endif
#ifndef ES_F32_U
#define ES_F32_U 3
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

template <int DT>
static cudaError_t launch_sum_t(const SumArgs& a, int max_ctas, cudaStream_t stream, int* grid_out,
                                bool launch = true) {
  if constexpr (DT == BF16 && ES_BF16_FFMA != 0) return launch_sum_bf16(a, max_ctas, stream, grid_out, launch);
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
  if constexpr (Cfg::TMA) fn = (const void*)sum_kernel_tma<DT, Cfg::C, Cfg::TU, Cfg::S, D>;
  else fn = (const void*)sum_kernel<DT, Cfg::T, Cfg::U, D>;
  static std::atomic<bool> configured[64] = {};  // idempotent set-up; atomic for concurrent first calls
  cudaError_t e = configure_once(fn, SMEM, configured);
  if (e != cudaSuccess || !launch) return e;
  // at least two vectors per column per CTA, at most one CTA per SM
  const int64_t want = (a.nvec + 2 * COLS - 1) / (2 * COLS);
  const int grid = (int)(want < 1 ? 1 : (want > max_ctas ? max_ctas : want));
  if (grid_out) *grid_out = grid;
  if constexpr (Cfg::TMA)
    return launch_single_array(sum_kernel_tma<DT, Cfg::C, Cfg::TU, Cfg::S, D>, grid, THREADS, SMEM, stream, a);
  else
    return launch_single_array(sum_kernel<DT, Cfg::T, Cfg::U, D>, grid, THREADS, SMEM, stream, a);
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
