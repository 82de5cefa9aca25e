/*
 * exactsum.h -- C ABI of the GB300 exact floating-point summation library.
 *
 * The library computes the exact sum of n IEEE floating-point values and
 * rounds it once, following Goodrich & Eldawy, "Parallel Algorithms for
 * Summing Floating-Point Numbers" (arXiv:1605.05436):
 *
 *   - the problem (Section 1): given X = {x_1..x_n}, return S_n*, a
 *     faithful rounding of S_n = sum x_i.  This library returns the
 *     correctly rounded value (round to nearest, ties to even, by default),
 *     which is always faithful, or a directed rounding on request;
 *   - the method (Sections 2, 3 and 5): convert each element into digits of
 *     a carry-free (alpha, beta)-regularised superaccumulator (Section 2,
 *     Lemma 1), add the digits without propagating carries, merge the
 *     partial accumulators carry-free, then propagate the signed carries
 *     once and round from the most significant non-zero digit (Section 3,
 *     steps 6-7; Section 5, steps 4-5).  The whole accumulator stays in
 *     on-chip memory and the input is streamed once (Section 5, Theorem 5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Element types: EXACTSUM_F64 (IEEE binary64), EXACTSUM_F32 (binary32),
 *    EXACTSUM_BF16 (bfloat16).  Arrays hold the raw IEEE bit patterns in
 *    the machine's (little-endian) order and must be aligned to their
 *    element size.  Subnormals are exact inputs.
 *  - Any input format may be rounded to any output format; the exact sum
 *    is rounded once, directly to the output format (no double rounding).
 *  - Special values (the paper is silent; these are the library's rules):
 *      any NaN, or both +Inf and -Inf present -> the quiet NaN of the output
 *        format with sign +, payload not preserved;
 *      otherwise any +Inf -> +Inf; otherwise any -Inf -> -Inf;
 *      otherwise the exact finite sum is rounded; overflow follows IEEE 754
 *        for the mode (to nearest -> Inf; toward zero -> max finite; up and
 *        down -> Inf on their side, max finite on the other).
 *  - Signed zero: an empty input gives +0.  If the exact sum is zero and
 *    n >= 1: all inputs -0 -> -0; all inputs +0 -> +0; otherwise -0 under
 *    EXACTSUM_RDOWN and +0 under the other modes (IEEE 754 rules for x + y).
 *  - Device pointers (prefix d_) are CUDA device memory owned by the
 *    caller; host pointers (prefix h_) are host memory owned by the caller
 *    (page-locked memory gives full copy bandwidth).  The library never
 *    frees caller memory.
 *  - Asynchrony: entry points that take a stream enqueue work on it and
 *    return without waiting, unless stated otherwise.  Results in device
 *    memory are valid once the stream has reached the call.
 *  - A handle (exactsum_t) owns device workspace.  Work enqueued through one
 *    handle must not overlap in time on the GPU: issue it on one stream, or
 *    order the streams.  Use one handle per concurrent stream.  A handle is
 *    not thread-safe; lock it or give each host thread its own.
 *  - Errors: every entry point returns an exactsum_status; no exception or
 *    abort crosses the ABI.  Arguments are checked on the host before any
 *    work is enqueued: a non-OK return means nothing was enqueued (except
 *    EXACTSUM_ECUDA, which reports a CUDA error from the launch or copy).
 *    exactsum_last_error() gives a message for the last failure.
 *  - Limits: n < 2^48 elements per call.
 */
#ifndef EXACTSUM_H
#define EXACTSUM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
/* A CUDA stream.  This is the very type of the CUDA runtime's cudaStream_t
 * (and of the driver's CUstream), declared here so that the header needs no
 * CUDA include: a cudaStream_t converts to it without a cast.  NULL is the
 * legacy default stream. */
typedef struct CUstream_st* exactsum_stream_t;

typedef struct exactsum_ctx* exactsum_t;

/* Element formats and rounding modes.  Both enums are passed as 32-bit
 * integers; the *_MAX_ENUM entries are not values, they only fix the enums'
 * range to the full 32-bit width so that an out-of-range argument reaches
 * the library's check (EXACTSUM_EINVAL) instead of being undefined. */
typedef enum {
    EXACTSUM_F64 = 0,   /* IEEE 754 binary64 */
    EXACTSUM_F32 = 1,   /* IEEE 754 binary32 */
    EXACTSUM_BF16 = 2,  /* bfloat16 (the upper half of a binary32) */
    EXACTSUM_DTYPE_MAX_ENUM = 0x7FFFFFFF
} exactsum_dtype;

typedef enum {
    EXACTSUM_RNE = 0,   /* to nearest, ties to even */
    EXACTSUM_RTZ = 1,   /* toward zero */
    EXACTSUM_RUP = 2,   /* toward +infinity */
    EXACTSUM_RDOWN = 3, /* toward -infinity */
    EXACTSUM_ROUND_MAX_ENUM = 0x7FFFFFFF
} exactsum_round;

typedef enum {
    EXACTSUM_OK = 0,
    EXACTSUM_EINVAL = 1,       /* bad argument (null, negative size, unknown enum,
                                  misaligned pointer, size over the limit) */
    EXACTSUM_ENOMEM = 2,       /* device or host allocation failed */
    EXACTSUM_ECUDA = 3,        /* a CUDA call failed; see exactsum_last_error */
    EXACTSUM_ETIMEOUT = 4,     /* a bounded wait gave up */
    EXACTSUM_EUNSUPPORTED = 5  /* device is not sm_103 */
} exactsum_status;

/* Words of an accumulator (see exactsum_acc_*): 72 signed 64-bit digits in
 * radix 2^32 (digit i weighs 2^(32 i) units of the input format's smallest
 * subnormal), then 5 counters (NaN seen, +Inf seen, -Inf seen, an element
 * other than +0 seen, an element other than -0 seen), then the element
 * count, then 2 reserved words.  Two accumulators of the same input format
 * merge by adding them word by word (Lemma 1: digit sums stay exact and
 * carries are deferred), so they can be summed across streams, devices or
 * processes with any integer all-reduce. */
#define EXACTSUM_ACC_DIGITS 72
#define EXACTSUM_ACC_WORDS 80
#define EXACTSUM_ACC_BYTES (EXACTSUM_ACC_WORDS * 8)

/* ---------------------------------------------------------------------- */
/* Handle                                                                  */
/* ---------------------------------------------------------------------- */

/* A handle serves every call below that computes the problem of Section 1
 * (given X = {x_1..x_n}, return a rounding of S_n = sum x_i): it owns the
 * workspace in which the reducers' partial accumulators meet before the
 * single post-process rounding (Section 6.1), so that no call allocates.
 *
 * Create a handle on CUDA device `device` (which becomes current on the
 * calling thread) and allocate its workspace.  `max_segments_hint` sizes
 * the segmented-sum workspace up front (0: grow on first use; growth
 * happens outside any stream capture).  On success *out receives the
 * handle.  Fails with EXACTSUM_EUNSUPPORTED on a device that is not
 * compute capability 10.3. */
exactsum_status exactsum_create(exactsum_t* out, int device, int64_t max_segments_hint);

/* Free the handle's workspace (after synchronising its device; Section 1
 * problem statement, as for exactsum_create).  NULL is OK. */
exactsum_status exactsum_destroy(exactsum_t h);

/* Message for the last failing call on `h` (or on a NULL handle); never
 * NULL; valid until the next call on the same handle. */
const char* exactsum_last_error(exactsum_t h);

/* ---------------------------------------------------------------------- */
/* Single array (Section 5 Theorem 5 shape: stream once, accumulator on    */
/* chip; Section 6.1 shape: each CTA a reducer, one post-process)          */
/* ---------------------------------------------------------------------- */

/* d_result (one element of out_dtype, device) <- round(sum of d_x[0..n)).
 * d_x: n elements of in_dtype in device memory (may be NULL when n == 0).
 * One kernel launch; no host synchronisation.  Results are stream-ordered
 * as usual; on the device, an FP64 call may start streaming its input while
 * the FP64 call just before it on the same stream (and handle) finishes its
 * merge (programmatic dependent launch: it waits for that call before it
 * touches the handle's workspace or its own result).  With any other stream
 * operation in between (a copy, an event, another kernel) the calls are
 * ordered as usual. */
exactsum_status exactsum_sum(exactsum_t h, const void* d_x, int64_t n, exactsum_dtype in_dtype,
                             exactsum_dtype out_dtype, exactsum_round mode, void* d_result, exactsum_stream_t stream);

/* End-to-end variant with host buffers: copies h_x to the device in
 * pipelined chunks on `stream`, sums it, copies the rounded result to
 * h_result (one element of out_dtype), and waits for the stream.  The
 * device copy buffers belong to the handle. */
exactsum_status exactsum_sum_host(exactsum_t h, const void* h_x, int64_t n, exactsum_dtype in_dtype,
                                  exactsum_dtype out_dtype, exactsum_round mode, void* h_result,
                                  exactsum_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Condition-number-sensitive sum (Section 4: r-truncated sparse           */
/* superaccumulators, r <- r^2 until a stopping condition holds; Section 2: */
/* sparse and gamma-truncated superaccumulators)                           */
/* ---------------------------------------------------------------------- */

/* d_result (one element of out_dtype, device) <- the same correctly rounded
 * sum as exactsum_sum, computed adaptively: pass r (r = 2, 4, 16) keeps in
 * every thread only the r most significant radix-2^32 digits of its running
 * sum, counts everything it drops and bounds it by B; the pass stops the
 * iteration when S - B, S and S + B round to the same value (S the sum of
 * the truncated partial sums), which then is the rounded exact sum.  When
 * r reaches the digits the format can occupy (67 FP64, 10 FP32, 9 BF16), the
 * exact single-pass kernel runs instead (nothing would be truncated).
 * Work is one pass over d_x per r tried: one pass for well-conditioned
 * inputs, up to four (FP64) for ill-conditioned ones.
 *
 * Synchronous: the host reads each pass's stopping flag, so the call
 * returns after the result is written (it synchronises `stream`).
 * passes (host, may be null) <- passes made (>= 1); last_r (host, may be
 * null) <- r of the pass that stopped, 0 if the exact kernel ran.  Errors
 * as for exactsum_sum; the handle's per-pass state (64 bytes of device and
 * page-locked host memory) is allocated on first use. */
exactsum_status exactsum_sum_adaptive(exactsum_t h, const void* d_x, int64_t n, exactsum_dtype in_dtype,
                                      exactsum_dtype out_dtype, exactsum_round mode, void* d_result, int* passes,
                                      int* last_r, exactsum_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Accumulators: exact partial sums that persist between calls             */
/* (Section 2: superaccumulator addition; Section 6.1: reducers write      */
/* partial accumulators that a post-process merges and rounds)             */
/* ---------------------------------------------------------------------- */

/* Set the EXACTSUM_ACC_WORDS words at d_acc (device, 8-byte aligned) to
 * zero (the empty sum). */
exactsum_status exactsum_acc_zero(exactsum_t h, void* d_acc, exactsum_stream_t stream);

/* d_acc += exact sum of d_x[0..n) (in_dtype).  All adds into one
 * accumulator must use the same in_dtype.  The digits are regularised
 * after each call (|digit| <= 2^32), so up to 2^30 accumulators can be
 * merged by plain addition. */
exactsum_status exactsum_acc_add(exactsum_t h, const void* d_x, int64_t n, exactsum_dtype in_dtype,
                                 void* d_acc, exactsum_stream_t stream);

/* d_result (one element of out_dtype) <- round(value of d_acc), where d_acc
 * holds sums of in_dtype elements.  d_acc is not modified. */
exactsum_status exactsum_acc_round(exactsum_t h, const void* d_acc, exactsum_dtype in_dtype,
                                   exactsum_dtype out_dtype, exactsum_round mode, void* d_result,
                                   exactsum_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Segmented (batched) sums: one launch for many CSR segments              */
/* (Section 6.1 MapReduce: tiles of the input are mapped to reducers,       */
/* each reducer builds an accumulator, per-key accumulators are merged     */
/* carry-free and rounded once)                                            */
/* ---------------------------------------------------------------------- */

/* Device status bits reported by exactsum_device_status. */
#define EXACTSUM_STATUS_BAD_OFFSETS 1  /* a segment had offsets[s+1] < offsets[s] or offsets[s] < 0 */
#define EXACTSUM_STATUS_MAP_OVERFLOW 2 /* more tiles than the tile map holds (input larger than HBM) */
#define EXACTSUM_STATUS_TIMEOUT 4      /* a bounded wait inside a kernel gave up; that result is invalid */

/* Diagnostic of the bounded waits (no paper counterpart).  Every wait
 * inside this library's kernels polls its mbarrier a bounded number of
 * times; if the phase has not completed by then the kernel sets
 * EXACTSUM_STATUS_TIMEOUT in the handle's device status word, waits
 * (bounded) for its own copies in flight and returns, so that the CUDA
 * context stays usable and the host learns of the failure from
 * exactsum_device_status.  This call runs that path on purpose: one thread
 * waits on an mbarrier that nothing ever completes, polling it `polls`
 * times (0: the kernels' own limit, through their own wait function), then
 * records EXACTSUM_STATUS_TIMEOUT.
 *   d_elapsed_ns: one uint64 in device memory (8-byte aligned) that receives
 *     the wait's duration in nanoseconds, or NULL.
 * Asynchronous on `stream`.  Errors: EXACTSUM_EINVAL for a null handle or a
 * misaligned d_elapsed_ns (nothing enqueued); EXACTSUM_ECUDA for a failed
 * launch. */
exactsum_status exactsum_check_timeout(exactsum_t h, uint32_t polls, uint64_t* d_elapsed_ns,
                                       exactsum_stream_t stream);

/* d_results[s] <- round(sum of d_x[d_offsets[s] .. d_offsets[s+1])) for
 * s in [0, num_segments).
 *   d_offsets: num_segments + 1 int64 CSR offsets in device memory (any
 *     non-decreasing, non-negative sequence; offsets[0] need not be 0).
 *   d_results: num_segments elements of out_dtype in device memory.
 * Empty segments give +0.  Segments with invalid offsets give a quiet NaN
 * and set EXACTSUM_STATUS_BAD_OFFSETS in the handle's device status word.
 * The work (a small planning pass plus one persistent reducer kernel) is
 * captured into a CUDA graph on first use of each (pointers, sizes, types,
 * configuration) signature and replayed afterwards; when `stream` is being
 * captured by the caller the kernels are launched into that capture instead.
 * The reducer configuration comes from the autotuner's table (see
 * exactsum_segmented_autotune) for this input format and size class
 * (ceil(log2 num_segments)), else a default.  Workspace grows on demand
 * (never during a capture); num_segments < 2^31. */
exactsum_status exactsum_segmented_sum(exactsum_t h, const void* d_x, const int64_t* d_offsets,
                                       int64_t num_segments, exactsum_dtype in_dtype, exactsum_dtype out_dtype, exactsum_round mode,
                                       void* d_results, exactsum_stream_t stream);

/* The one-launch-per-segment form of the same computation: h_offsets are
 * in host memory and every segment is summed by its own exactsum_sum call.
 * Same results bit for bit; kept as the baseline the batched call is
 * measured against. */
exactsum_status exactsum_sum_each(exactsum_t h, const void* d_x, const int64_t* h_offsets,
                                  int64_t num_segments, exactsum_dtype in_dtype, exactsum_dtype out_dtype, exactsum_round mode,
                                  void* d_results, exactsum_stream_t stream);

/* Autotuner (synchronous): times each reducer configuration on this very
 * input -- the register-streaming reducer with two CTA sizes, the
 * TMA-ring reducer (kind 1) and the windowed reducer (kind 2: narrow
 * per-lane digit windows plus an exact overflow accumulator, fast when a
 * tile's exponents are concentrated), each with three tile sizes -- keeps
 * the fastest for the input format and size class, and reports it through
 * the non-NULL output pointers (kind: 0 register streaming, 1 TMA ring,
 * 2 windowed).
 * d_results_scratch: num_segments elements of in_dtype. */
exactsum_status exactsum_segmented_autotune(exactsum_t h, const void* d_x, const int64_t* d_offsets,
                                            int64_t num_segments, exactsum_dtype in_dtype,
                                            void* d_results_scratch, exactsum_stream_t stream,
                                            int* best_warps, int* best_kind, int64_t* best_tile,
                                            float* best_ms);

/* Save / load the autotuner's table as JSON
 * ({"segmented": [{"in_dtype", "log2_segments", "warps", "kind", "tile", "ms"}...]}). */
exactsum_status exactsum_tuning_save(exactsum_t h, const char* path);
exactsum_status exactsum_tuning_load(exactsum_t h, const char* path);

/* Synchronise the handle's device, return the accumulated device status
 * bits (EXACTSUM_STATUS_*) in *status_out and clear them. */
exactsum_status exactsum_device_status(exactsum_t h, int64_t* status_out);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of exact-sum requests                      */
/* (no paper counterpart: the reducer state of Section 6.1 kept on the     */
/* device while requests of mixed sizes come and go)                       */
/* ---------------------------------------------------------------------- */

typedef struct exactsum_server* exactsum_server_t;

/* One finished request, as reported by exactsum_server_poll. */
typedef struct {
    uint64_t id;           /* from exactsum_server_submit */
    int32_t status;        /* EXACTSUM_OK; EXACTSUM_ENOMEM if staging memory could not be
                              allocated; EXACTSUM_ECUDA if the engine failed */
    int32_t out_dtype;
    uint64_t result_bits;  /* the rounded sum in the low 16/32/64 bits */
    int64_t n;
    int64_t submit_ns;     /* exactsum_server_clock_ns() at submission, */
    int64_t admit_ns;      /* at admission into a slot, */
    int64_t done_ns;       /* when the result was visible on the host */
} exactsum_completion;

/* Start a serving engine on `device` with its own streams and a scheduler
 * thread.
 *   max_slots (1..256): requests resident at once; each owns one device
 *     accumulator slot for its whole life, across steps.
 *   mem_budget_bytes: admission limit on the bytes held by resident
 *     requests (input bytes + EXACTSUM_ACC_BYTES each).  A request waits,
 *     in arrival order, until a slot is free and the budget has room; a
 *     request larger than the whole budget is admitted alone.
 *   chunk_elems: elements of each request processed per step (continuous
 *     batching: every step carries one chunk of every resident request, in
 *     one kernel, so requests that arrive later join at the next step).
 *   tile_elems: largest warp work unit in elements (multiple of 64 dividing
 *     chunk_elems); a chunk is cut into tiles of about chunk / (warps of the
 *     step kernel), whole multiples of 1,024 elements, at least 2,048 and at
 *     most tile_elems, so that every chunk is spread over the whole GPU.
 *   max_steps_per_request: if > 0, a request's chunk grows to
 *     ceil(n / max_steps_per_request) (whole tiles) when that is larger than
 *     chunk_elems, so that no request needs more than that many steps; 0
 *     keeps the fixed chunk. */
exactsum_status exactsum_server_create(exactsum_server_t* out, int device, int max_slots,
                                       int64_t mem_budget_bytes, int64_t chunk_elems,
                                       int64_t tile_elems, int max_steps_per_request);

/* Queue a request: the exact sum of x[0..n) (in_dtype) rounded to
 * out_dtype under mode.  x_on_host = 0: x is device memory that must stay
 * valid and unchanged until the request completes.  x_on_host = 1: x is
 * host memory (page-locked for speed); the engine copies it to the device
 * after admission, and x must stay valid until completion.  Thread-safe;
 * returns at once with the request id in *id_out. */
exactsum_status exactsum_server_submit(exactsum_server_t s, const void* x, int64_t n, exactsum_dtype in_dtype,
                                       exactsum_dtype out_dtype, exactsum_round mode, int x_on_host, uint64_t* id_out);

/* Move up to max_out completion records into out; *count receives how many. */
exactsum_status exactsum_server_poll(exactsum_server_t s, exactsum_completion* out, int max_out,
                                     int* count);

/* Wait until every submitted request has completed (EXACTSUM_ETIMEOUT after
 * timeout_ms milliseconds). */
exactsum_status exactsum_server_drain(exactsum_server_t s, int64_t timeout_ms);

/* Lanes (call before the first exactsum_server_submit; EXACTSUM_EINVAL
 * afterwards).  A request whose input exceeds express_max_bytes takes the
 * bulk lane: one launch of the single-array sum kernel (exactsum_sum's) on
 * all SMs but express_sms, its result rounded straight into pinned host
 * memory.  Smaller requests take the express lane, on the SMs the bulk lane
 * leaves free, so that they never wait behind a large request:
 *   resident = 1 (default): a resident kernel on express_sms SMs takes each
 *     request from a ring in pinned host memory as soon as it is admitted
 *     (no launch per request); its tiles are summed by whichever warps are
 *     free, with the tiles of all requests in flight interleaved (continuous
 *     batching at tile granularity), and the warp that finishes a request's
 *     last tile rounds it and publishes the result.  The kernel leaves
 *     after 5 ms without work and is launched again by the next request;
 *     while it runs, those SMs are busy polling, so other kernels of the
 *     process get the remaining SMs.  (With CUDA's lazy module loading, a
 *     kernel launched for the first time in the process waits for the
 *     kernels already running: exactsum_server_create therefore loads all
 *     of this library's kernels; other code that launches a kernel for the
 *     first time while the resident kernel runs waits until requests pause
 *     for 5 ms, unless the process loads modules eagerly,
 *     CUDA_MODULE_LOADING=EAGER);
 *   resident = 0: continuous-batching steps (one kernel launch per step,
 *     carrying a chunk of every express request in flight) on the free SMs
 *     (all SMs while no bulk launch is in flight).
 * Defaults: 4 MiB, 8 SMs, resident.  express_max_bytes < 0 sends every
 * request to the express lane; express_sms must be in [1, SMs). */
exactsum_status exactsum_server_set_lanes(exactsum_server_t s, int64_t express_max_bytes, int express_sms,
                                         int resident);

/* Counters: steps launched, most requests resident at once, requests not yet complete. */
exactsum_status exactsum_server_stats(exactsum_server_t s, int64_t* steps, int64_t* peak_active,
                                      int64_t* outstanding);

/* The engine's steady clock, in nanoseconds. */
int64_t exactsum_server_clock_ns(void);

/* Message for the server's last failure. */
const char* exactsum_server_last_error(exactsum_server_t s);

/* Finish every request still in the system, stop the scheduler and free
 * the engine. */
exactsum_status exactsum_server_destroy(exactsum_server_t s);

/* ---------------------------------------------------------------------- */
/* Allocation-free segmented sum                                           */
/* (no counterpart in the paper: a deployment variant of                   */
/* exactsum_segmented_sum)                                                 */
/* ---------------------------------------------------------------------- */

#define EXACTSUM_NOALLOC_MAX_SEGMENTS 2048

/* The same results as exactsum_segmented_sum, for callers that cannot
 * allocate device memory -- a plug-in whose host application owns all device
 * memory through its own pool or allocator, a program that must keep a fixed
 * memory footprint, a real-time host that forbids allocation after start-up.
 * Such callers cannot create a handle (exactsum_create allocates its
 * workspace).  This call needs no handle and calls no cudaMalloc, cudaFree
 * or other allocating routine: its scratch is one fixed array of about
 * 3.4 MB in the library's own device memory, present on every GPU that loads
 * the library until the process exits.  (The paper has no counterpart: this
 * is a deployment variant of exactsum_segmented_sum.)
 *   - Runs on the calling thread's current device; arguments as in
 *     exactsum_segmented_sum (device input, device int64 offsets, device
 *     results).
 *   - num_segments must not exceed EXACTSUM_NOALLOC_MAX_SEGMENTS; a larger
 *     call returns EXACTSUM_EINVAL (message in exactsum_last_error(NULL))
 *     and enqueues nothing.  Inputs up to 512 GiB are covered.
 *   - Invalid offsets (offsets[s+1] < offsets[s] or offsets[s] < 0) give a
 *     quiet NaN for that segment; no status word is reported (there is no
 *     handle to read it through), so check offsets beforehand when a NaN
 *     result must mean NaN data.
 *   - All calls share the one scratch array and each call clears the parts
 *     that must start at zero: calls whose work overlaps on the GPU race,
 *     so order them (for example on one stream).
 *   - The first call on each device looks up the scratch array's device
 *     address and keeps it for the life of the process; make that first
 *     call before any stream capture starts, and do not use this entry point
 *     after cudaDeviceReset on that device (the kept address would be
 *     stale).
 *   - Asynchronous on `stream`. */
exactsum_status exactsum_segmented_sum_noalloc(const void* d_x, const int64_t* d_offsets,
                                               int64_t num_segments, exactsum_dtype in_dtype, exactsum_dtype out_dtype,
                                               exactsum_round mode, void* d_results, exactsum_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* EXACTSUM_H */
