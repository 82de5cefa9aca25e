/*
 * abi_example.c -- the C ABI used from plain C (C99, no C++), as a user of
 * include/exactsum.h would: create a handle, sum device arrays, a segmented
 * sum, read the results, destroy.  Built and run by tests/test_c_abi.py.
 *
 *   abi_example nogpu   with no usable GPU: exactsum_create must fail with a
 *                       status and a message, and nothing may crash
 *   abi_example gpu     on a GB300: the sums must be the exact ones
 */
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include "exactsum.h"

static int fail(const char* what, exactsum_t h) {
    printf("FAIL %s: %s\n", what, exactsum_last_error(h));
    return 1;
}

int main(int argc, char** argv) {
    exactsum_t h = NULL;
    exactsum_status st = exactsum_create(&h, 0, 16);
    if (argc > 1 && strcmp(argv[1], "nogpu") == 0) {
        if (st == EXACTSUM_OK) {
            exactsum_destroy(h);
            printf("FAIL create succeeded without a GPU\n");
            return 1;
        }
        printf("OK no GPU: status %d: %s\n", (int)st, exactsum_last_error(NULL));
        return 0;
    }
    if (st != EXACTSUM_OK) return fail("create", NULL);

    /* 1 + 2 + ... + 1000 = 500500 exactly; then 1e300 + 1 - 1e300 = 1 */
    double hx[1003];
    for (int i = 0; i < 1000; ++i) hx[i] = (double)(i + 1);
    hx[1000] = 1e300;
    hx[1001] = 1.0;
    hx[1002] = -1e300;
    int64_t hoff[3] = {0, 1000, 1003};
    double *dx = NULL, *dres = NULL;
    int64_t* doff = NULL;
    if (cudaMalloc((void**)&dx, sizeof hx) != cudaSuccess || cudaMalloc((void**)&dres, 3 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&doff, sizeof hoff) != cudaSuccess)
        return fail("cudaMalloc", h);
    cudaMemcpy(dx, hx, sizeof hx, cudaMemcpyHostToDevice);
    cudaMemcpy(doff, hoff, sizeof hoff, cudaMemcpyHostToDevice);
    cudaStream_t s = NULL;  /* a cudaStream_t is an exactsum_stream_t */
    if (exactsum_sum(h, dx, 1000, EXACTSUM_F64, EXACTSUM_F64, EXACTSUM_RNE, dres, s) != EXACTSUM_OK)
        return fail("sum", h);
    if (exactsum_segmented_sum(h, dx, doff, 2, EXACTSUM_F64, EXACTSUM_F64, EXACTSUM_RNE, dres + 1, s) != EXACTSUM_OK)
        return fail("segmented_sum", h);
    /* an unknown format is refused before anything is enqueued */
    if (exactsum_sum(h, dx, 1000, (exactsum_dtype)7, EXACTSUM_F64, EXACTSUM_RNE, dres, s) != EXACTSUM_EINVAL)
        return fail("unknown dtype accepted", h);
    double r[3];
    cudaMemcpy(r, dres, sizeof r, cudaMemcpyDeviceToHost);
    if (r[0] != 500500.0 || r[1] != 500500.0 || r[2] != 1.0) {
        printf("FAIL results %.17g %.17g %.17g\n", r[0], r[1], r[2]);
        return 1;
    }
    cudaFree(dx);
    cudaFree(dres);
    cudaFree(doff);
    if (exactsum_destroy(h) != EXACTSUM_OK) return fail("destroy", NULL);
    printf("OK %.17g %.17g %.17g\n", r[0], r[1], r[2]);
    return 0;
}
