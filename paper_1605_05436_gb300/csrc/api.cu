// api.cu -- the C ABI (include/exactsum.h): handle, argument checks, launches.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/exactsum.h"
#include "digits.cuh"
#include "internal.h"
#include "handle.h"

using es::ACC_WORDS;

static thread_local std::string g_null_handle_error = "no error";

static exactsum_status fail(exactsum_t h, exactsum_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->last_error = buf;
  else g_null_handle_error = buf;
  return st;
}

// Message for entry points that have no handle (reported by
// exactsum_last_error(NULL) on the calling thread).
void es_set_detached_error(const char* msg) { g_null_handle_error = msg; }

exactsum_status es_cuda_fail(exactsum_t h, cudaError_t e, const char* what) {
  return fail(h, EXACTSUM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static bool valid_dtype(int d) { return d == EXACTSUM_F64 || d == EXACTSUM_F32 || d == EXACTSUM_BF16; }
static bool valid_mode(int m) { return m >= EXACTSUM_RNE && m <= EXACTSUM_RDOWN; }
static int elem_bytes(int d) { return d == EXACTSUM_F64 ? 8 : (d == EXACTSUM_F32 ? 4 : 2); }
static constexpr int64_t MAX_N = (int64_t)1 << 48;

exactsum_status es_check_common(exactsum_t h, const void* x, int64_t n, int in, int out, int mode,
                                const void* dst) {
  if (!h) return fail(h, EXACTSUM_EINVAL, "null handle");
  if (!valid_dtype(in)) return fail(h, EXACTSUM_EINVAL, "unknown input dtype %d", in);
  if (out >= 0 && !valid_dtype(out)) return fail(h, EXACTSUM_EINVAL, "unknown output dtype %d", out);
  if (mode >= 0 && !valid_mode(mode)) return fail(h, EXACTSUM_EINVAL, "unknown rounding mode %d", mode);
  if (n < 0 || n >= MAX_N) return fail(h, EXACTSUM_EINVAL, "n = %lld out of range [0, 2^48)", (long long)n);
  if (n > 0 && !x) return fail(h, EXACTSUM_EINVAL, "null input with n > 0");
  if (((uintptr_t)x) % elem_bytes(in)) return fail(h, EXACTSUM_EINVAL, "input not aligned to its element size");
  if (!dst) return fail(h, EXACTSUM_EINVAL, "null output");
  return EXACTSUM_OK;
}

static exactsum_status set_device(exactsum_t h) {
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return es_cuda_fail(h, e, "cudaSetDevice");
  return EXACTSUM_OK;
}

extern "C" {

exactsum_status exactsum_create(exactsum_t* out, int device, int64_t max_segments_hint) {
  if (!out) return fail(nullptr, EXACTSUM_EINVAL, "null output handle pointer");
  *out = nullptr;
  if (max_segments_hint < 0) return fail(nullptr, EXACTSUM_EINVAL, "negative segment hint");
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return fail(nullptr, EXACTSUM_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  if (device < 0 || device >= count) return fail(nullptr, EXACTSUM_EINVAL, "device %d not present", device);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return fail(nullptr, EXACTSUM_ECUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
  if (prop.major != 10 || prop.minor != 3)
    return fail(nullptr, EXACTSUM_EUNSUPPORTED, "device %d is sm_%d%d; this build targets sm_103a",
                device, prop.major, prop.minor);
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(nullptr, EXACTSUM_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  exactsum_t h = new (std::nothrow) exactsum_ctx();
  if (!h) return fail(nullptr, EXACTSUM_ENOMEM, "host allocation failed");
  h->device = device;
  h->num_sms = prop.multiProcessorCount;
  h->max_ctas = h->num_sms;
  exactsum_status st = es_workspace_init(h);
  if (st == EXACTSUM_OK && max_segments_hint > 0) st = es_segment_workspace_reserve(h, max_segments_hint);
  if (st != EXACTSUM_OK) {
    g_null_handle_error = h->last_error;
    es_workspace_free(h);
    delete h;
    return st;
  }
  *out = h;
  return EXACTSUM_OK;
}

exactsum_status exactsum_destroy(exactsum_t h) {
  if (!h) return EXACTSUM_OK;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  es_workspace_free(h);
  delete h;
  return EXACTSUM_OK;
}

const char* exactsum_last_error(exactsum_t h) {
  return h ? h->last_error.c_str() : g_null_handle_error.c_str();
}

exactsum_status exactsum_sum(exactsum_t h, const void* d_x, int64_t n, exactsum_dtype in_dtype, exactsum_dtype out_dtype,
                             exactsum_round mode, void* d_result, exactsum_stream_t stream) {
  exactsum_status st = es_check_common(h, d_x, n, in_dtype, out_dtype, mode, d_result);
  if (st != EXACTSUM_OK) return st;
  if ((st = set_device(h)) != EXACTSUM_OK) return st;
  es::SumArgs a = es_make_sum_args(d_x, n, in_dtype);
  a.out = out_dtype;
  a.mode = mode;
  a.result = d_result;
  a.acc = nullptr;
  a.partials = h->partials;
  a.ticket = h->ticket;
  a.status = h->dev_status;
  cudaError_t e = es::launch_sum(in_dtype, a, h->max_ctas, (cudaStream_t)stream, nullptr);
  if (e != cudaSuccess) return es_cuda_fail(h, e, "sum kernel launch");
  return EXACTSUM_OK;
}

exactsum_status exactsum_acc_zero(exactsum_t h, void* d_acc, exactsum_stream_t stream) {
  if (!h) return fail(h, EXACTSUM_EINVAL, "null handle");
  if (!d_acc || ((uintptr_t)d_acc) % 8) return fail(h, EXACTSUM_EINVAL, "accumulator must be non-null and 8-byte aligned");
  exactsum_status st = set_device(h);
  if (st != EXACTSUM_OK) return st;
  cudaError_t e = cudaMemsetAsync(d_acc, 0, EXACTSUM_ACC_BYTES, (cudaStream_t)stream);
  if (e != cudaSuccess) return es_cuda_fail(h, e, "cudaMemsetAsync");
  return EXACTSUM_OK;
}

exactsum_status exactsum_acc_add(exactsum_t h, const void* d_x, int64_t n, exactsum_dtype in_dtype, void* d_acc,
                                 exactsum_stream_t stream) {
  exactsum_status st = es_check_common(h, d_x, n, in_dtype, -1, -1, d_acc);
  if (st != EXACTSUM_OK) return st;
  if (((uintptr_t)d_acc) % 8) return fail(h, EXACTSUM_EINVAL, "accumulator must be 8-byte aligned");
  if ((st = set_device(h)) != EXACTSUM_OK) return st;
  if (n == 0) return EXACTSUM_OK;
  es::SumArgs a = es_make_sum_args(d_x, n, in_dtype);
  a.out = in_dtype;
  a.mode = 0;
  a.result = nullptr;
  a.acc = (int64_t*)d_acc;
  a.partials = h->partials;
  a.ticket = h->ticket;
  a.status = h->dev_status;
  cudaError_t e = es::launch_sum(in_dtype, a, h->max_ctas, (cudaStream_t)stream, nullptr);
  if (e != cudaSuccess) return es_cuda_fail(h, e, "accumulate kernel launch");
  return EXACTSUM_OK;
}

exactsum_status exactsum_acc_round(exactsum_t h, const void* d_acc, exactsum_dtype in_dtype, exactsum_dtype out_dtype,
                                   exactsum_round mode, void* d_result, exactsum_stream_t stream) {
  exactsum_status st = es_check_common(h, d_acc, 1, in_dtype, out_dtype, mode, d_result);
  if (st != EXACTSUM_OK) return st;
  if (((uintptr_t)d_acc) % 8) return fail(h, EXACTSUM_EINVAL, "accumulator must be 8-byte aligned");
  if ((st = set_device(h)) != EXACTSUM_OK) return st;
  cudaError_t e = es::launch_round_acc((const int64_t*)d_acc, in_dtype, out_dtype, mode, d_result,
                                       (cudaStream_t)stream);
  if (e != cudaSuccess) return es_cuda_fail(h, e, "round kernel launch");
  return EXACTSUM_OK;
}

exactsum_status exactsum_sum_host(exactsum_t h, const void* h_x, int64_t n, exactsum_dtype in_dtype, exactsum_dtype out_dtype,
                                  exactsum_round mode, void* h_result, exactsum_stream_t stream) {
  exactsum_status st = es_check_common(h, h_x, n, in_dtype, out_dtype, mode, h_result);
  if (st != EXACTSUM_OK) return st;
  if ((st = set_device(h)) != EXACTSUM_OK) return st;
  return es_sum_host_pipelined(h, h_x, n, in_dtype, out_dtype, mode, h_result, (cudaStream_t)stream);
}

}  // extern "C"

es::SumArgs es_make_sum_args(const void* x, int64_t n, int in_dtype) {
  es::SumArgs a{};
  const int eb = elem_bytes(in_dtype);
  const int epv = 16 / eb;
  int64_t head = 0;
  if (n > 0) {
    const uintptr_t mis = ((uintptr_t)x) & 15u;
    head = mis ? (int64_t)((16 - mis) / eb) : 0;
    if (head > n) head = n;
  }
  a.x = x;
  a.n = n;
  a.head = head;
  a.nvec = (n - head) / epv;
  a.tail = n - head - a.nvec * epv;
  return a;
}
