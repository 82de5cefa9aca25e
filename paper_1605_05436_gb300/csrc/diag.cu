// diag.cu -- a diagnostic of the kernels' bounded waits.
//
// Every wait inside this library's kernels (on an mbarrier that a bulk copy
// or a consumer warp completes) polls a bounded number of times; when the
// phase has not completed by then, the kernel sets STATUS_TIMEOUT in the
// handle's device status word, waits (again bounded) for its own copies in
// flight and returns, so the CUDA context stays usable.  This file lets a
// caller or a test see that path run: one thread waits, with the same
// polling loop, on an mbarrier that nothing ever completes.
#include <cuda_runtime.h>

#include "../../include/exactsum.h"
#include "handle.h"
#include "internal.h"
#include "tma.cuh"

namespace es {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One thread initialises an mbarrier that expects one arrival, never
// arrives, and polls it `polls` times (0: the kernels' own limit, through
// the kernels' own wait function).
__global__ void bounded_wait_kernel(unsigned long long* status, uint32_t polls,
                                    unsigned long long* elapsed_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_init_fence();
  const unsigned long long t0 = global_ns();
  bool done = false;
  if (polls == 0) {
    done = mbar_wait(&bar, 0);
  } else {
    for (uint32_t i = 0; i < polls && !done; ++i) done = mbar_test_parity(&bar, 0);
  }
  const unsigned long long t1 = global_ns();
  if (!done) atomicOr(status, STATUS_TIMEOUT);
  if (elapsed_ns) *elapsed_ns = t1 - t0;
}

}  // namespace es

void es_set_detached_error(const char* msg);

extern "C" exactsum_status exactsum_check_timeout(exactsum_t h, uint32_t polls, uint64_t* d_elapsed_ns,
                                                  exactsum_stream_t stream) {
  if (!h) {
    es_set_detached_error("null handle");
    return EXACTSUM_EINVAL;
  }
  if (((uintptr_t)d_elapsed_ns) % 8) {
    h->last_error = "d_elapsed_ns must be 8-byte aligned";
    return EXACTSUM_EINVAL;
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return es_cuda_fail(h, e, "cudaSetDevice");
  es::bounded_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(h->dev_status, polls,
                                                             (unsigned long long*)d_elapsed_ns);
  if ((e = cudaGetLastError()) != cudaSuccess) return es_cuda_fail(h, e, "bounded-wait kernel launch");
  return EXACTSUM_OK;
}
