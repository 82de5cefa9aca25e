// noalloc.cu -- the segmented exact sum for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc at all: plug-ins whose host
// application owns all device memory through its own pool or allocator,
// programs that must keep a fixed memory footprint, and embedded or
// real-time hosts that forbid allocation after start-up.  They cannot create a handle
// (exactsum_create allocates its workspace), so this entry point keeps its
// scratch in one fixed-size array in the library's own device memory
// (g_noalloc_scratch below, about 3.4 MB on every GPU that loads the
// library, held until the process exits) and runs the same planner and
// reducer kernels as exactsum_segmented_sum on it.  It calls no cudaMalloc,
// no cudaFree and no allocating library routine.
//
// Limits and sharing:
//   - at most NOALLOC_MAX_SEGMENTS segments per call (larger calls are
//     rejected with EXACTSUM_EINVAL before anything is enqueued);
//   - tiles are 1 MiB of input, and the tile map holds enough entries for
//     inputs up to 512 GiB;
//   - every call uses the same array: calls whose work overlaps on the GPU
//     (different streams without ordering, or different host threads) race
//     and give wrong results; order them on one stream;
//   - the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current and keeps it for the
//     life of the process; make that first call before any stream capture
//     begins, and do not call this after cudaDeviceReset on that device;
//   - invalid offsets give NaN for their segment; the status word that
//     records them lives in the shared scratch and is not reported.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/exactsum.h"
#include "digits.cuh"
#include "internal.h"
#include "segmented.h"

void es_set_detached_error(const char* msg);

namespace {

constexpr int64_t NOALLOC_MAX_SEGMENTS = EXACTSUM_NOALLOC_MAX_SEGMENTS;
constexpr int64_t NOALLOC_TILE_BYTES = (int64_t)1 << 20;
constexpr int64_t NOALLOC_MAP_ENTRIES = NOALLOC_MAX_SEGMENTS + ((int64_t)1 << 19);

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
// byte offsets of the regions inside the scratch array
constexpr size_t OFF_ACC = 0;
constexpr size_t OFF_BASE = align256(OFF_ACC + (size_t)NOALLOC_MAX_SEGMENTS * es::ACC_WORDS * 8);
constexpr size_t OFF_REMAINING = align256(OFF_BASE + (size_t)(NOALLOC_MAX_SEGMENTS + 1) * 8);
constexpr size_t OFF_BLOCKS = align256(OFF_REMAINING + (size_t)NOALLOC_MAX_SEGMENTS * 4);
constexpr size_t OFF_MAP = align256(OFF_BLOCKS + (size_t)((NOALLOC_MAX_SEGMENTS + 1023) / 1024) * 8);
constexpr size_t OFF_COUNTERS = align256(OFF_MAP + (size_t)NOALLOC_MAP_ENTRIES * 4);
constexpr size_t OFF_STATUS = OFF_COUNTERS + 64;
constexpr size_t SCRATCH_BYTES = align256(OFF_STATUS + 64);

struct DeviceScratch {
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  int num_sms = 0;
};

std::mutex g_setup_mu;
DeviceScratch g_devices[64];

int elem_bytes(int d) { return d == EXACTSUM_F64 ? 8 : (d == EXACTSUM_F32 ? 4 : 2); }

exactsum_status reject(exactsum_status st, const char* msg) {
  es_set_detached_error(msg);
  return st;
}

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// symbol, not a device address: host code passes the address obtained from
// cudaGetSymbolAddress to the kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

// Once per device, with that device current: find the array's device
// address and the SM count.
exactsum_status setup(int dev, DeviceScratch* out) {
  std::lock_guard<std::mutex> g(g_setup_mu);
  DeviceScratch& d = g_devices[dev];
  if (!d.base) {
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return reject(EXACTSUM_ECUDA, "cudaGetDeviceProperties failed");
    if (prop.major != 10 || prop.minor != 3) return reject(EXACTSUM_EUNSUPPORTED, "this build targets sm_103a");
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      char msg[160];
      std::snprintf(msg, sizeof msg, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
      return reject(EXACTSUM_ECUDA, msg);
    }
    d.base = (unsigned char*)p;
    d.num_sms = prop.multiProcessorCount;
  }
  *out = d;
  return EXACTSUM_OK;
}

}  // namespace

extern "C" exactsum_status exactsum_segmented_sum_noalloc(const void* d_x, const int64_t* d_offsets,
                                                          int64_t num_segments, exactsum_dtype in_dtype,
                                                          exactsum_dtype out_dtype, exactsum_round mode, void* d_results,
                                                          exactsum_stream_t stream) {
  if (in_dtype < 0 || in_dtype > 2 || out_dtype < 0 || out_dtype > 2)
    return reject(EXACTSUM_EINVAL, "unknown dtype");
  if (mode < 0 || mode > 3) return reject(EXACTSUM_EINVAL, "unknown rounding mode");
  if (num_segments < 0) return reject(EXACTSUM_EINVAL, "negative num_segments");
  if (num_segments > NOALLOC_MAX_SEGMENTS) {
    char msg[200];
    std::snprintf(msg, sizeof msg,
                  "num_segments = %lld exceeds the allocation-free maximum of %lld segments per call",
                  (long long)num_segments, (long long)NOALLOC_MAX_SEGMENTS);
    return reject(EXACTSUM_EINVAL, msg);
  }
  if (num_segments > 0 && (!d_offsets || !d_results)) return reject(EXACTSUM_EINVAL, "null offsets or results");
  if (((uintptr_t)d_offsets) % 8) return reject(EXACTSUM_EINVAL, "offsets not 8-byte aligned");
  if (((uintptr_t)d_x) % elem_bytes(in_dtype)) return reject(EXACTSUM_EINVAL, "input not aligned to its element size");
  if (((uintptr_t)d_results) % elem_bytes(out_dtype)) return reject(EXACTSUM_EINVAL, "results not aligned");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return reject(EXACTSUM_ECUDA, "no current CUDA device");
  DeviceScratch ds;
  exactsum_status st = setup(dev, &ds);
  if (st != EXACTSUM_OK) return st;
  if (num_segments == 0) return EXACTSUM_OK;

  cudaStream_t s = (cudaStream_t)stream;
  // the per-segment accumulators and the status word must start at zero;
  // the planner rewrites every other region on each call
  cudaError_t e = cudaMemsetAsync(ds.base + OFF_ACC, 0, (size_t)num_segments * es::ACC_WORDS * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ds.base + OFF_STATUS, 0, 64, s);
  if (e != cudaSuccess) return reject(EXACTSUM_ECUDA, "cudaMemsetAsync(scratch) failed");

  es::SegArgs a{};
  a.x = d_x;
  a.off = d_offsets;
  a.S = num_segments;
  a.out = out_dtype;
  a.mode = mode;
  a.results = d_results;
  a.tile = NOALLOC_TILE_BYTES / elem_bytes(in_dtype);
  a.block_tiles = (int64_t*)(ds.base + OFF_BLOCKS);
  a.tile_base = (int64_t*)(ds.base + OFF_BASE);
  a.tile_seg = (int32_t*)(ds.base + OFF_MAP);
  a.map_capacity = NOALLOC_MAP_ENTRIES;
  a.remaining = (unsigned int*)(ds.base + OFF_REMAINING);
  a.seg_acc = (int64_t*)(ds.base + OFF_ACC);
  a.counters = (unsigned long long*)(ds.base + OFF_COUNTERS);
  a.status = (unsigned long long*)(ds.base + OFF_STATUS);
  e = es::seg_enqueue(in_dtype, a, es::seg_warps_choice(in_dtype, 0), es::SEG_KIND_REGISTER, ds.num_sms, s);
  if (e != cudaSuccess) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "segmented launch: %s", cudaGetErrorString(e));
    return reject(EXACTSUM_ECUDA, msg);
  }
  return EXACTSUM_OK;
}
