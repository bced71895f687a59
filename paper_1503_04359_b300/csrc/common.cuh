// Shared internals of libdobfs: status/error plumbing, the device allocator
// hook, launch geometry and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "../../include/dobfs.h"

namespace dobfs {

// ------------------------------------------------------------------ errors
// Thread-local last-error text plus a status code; every C entry point
// returns the code of the first failure it met.
int set_error(int status, const char* fmt, ...);
void clear_error();

#define DOBFS_CUDA_TRY(expr)                                                                   \
  do {                                                                                          \
    cudaError_t _e = (expr);                                                                    \
    if (_e != cudaSuccess) {                                                                    \
      return ::dobfs::set_error(DOBFS_ERR_CUDA, "%s failed at %s:%d: %s", #expr, __FILE__,      \
                                __LINE__, cudaGetErrorString(_e));                              \
    }                                                                                           \
  } while (0)

#define DOBFS_TRY(expr)        \
  do {                         \
    int _s = (expr);           \
    if (_s != DOBFS_OK) {      \
      return _s;               \
    }                          \
  } while (0)

// ------------------------------------------------------------------ memory
// All library-owned device memory goes through the process-wide allocator
// hook (default cudaMalloc/cudaFree).
void* dev_alloc(size_t bytes, cudaStream_t stream);
void dev_free(void* p, cudaStream_t stream);

// Owning device buffer; frees through the allocator hook.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : ptr(o.ptr), bytes(o.bytes), stream(o.stream) { o.ptr = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      reset();
      ptr = o.ptr; bytes = o.bytes; stream = o.stream;
      o.ptr = nullptr; o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { reset(); }
  int alloc(size_t n_bytes, cudaStream_t s);   // DOBFS_OK or DOBFS_ERR_OOM
  void reset();
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// true if p is device (or managed) memory reachable by kernels as a device pointer
bool is_device_ptr(const void* p);

// ------------------------------------------------------------------ geometry
int sm_count();
constexpr int kWarp = 32;

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline int bits_for(int64_t n) {  // smallest b with 2^b >= n (n >= 1)
  int b = 0;
  while ((int64_t(1) << b) < n) ++b;
  return b;
}

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Block-wide sum of a 64-bit value, result valid in thread 0. `sh` needs
// blockDim/32 slots.
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if (lane_id() == 0) sh[w] = v;
  __syncthreads();
  unsigned long long t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  __syncthreads();
  return t;
}

// ------------------------------------------------------------------ bounds-check builds
// Built with -DDOBFS_BOUNDS_CHECK, every index the kernels read from memory
// (a vertex ID from a column, queue, record or map; a row's offsets; a write
// position from a counter) is checked before use. A failing check records
// its site in the run's control block (the first site wins) and substitutes
// a safe value, so the access that follows stays in bounds; the host then
// fails the call with DOBFS_ERR_BOUNDS. In normal builds the checks compile
// away. Site numbers are listed in bounds_site_name().
#ifdef DOBFS_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif

// Bounds-check builds also over-allocate every device buffer by
// kBoundsSlackBytes, enough for kBoundsSlackVertices vertices past n in any
// per-vertex array, so that a corrupted vertex ID below n +
// kBoundsSlackVertices stays inside the allocation even at an access the
// checks would miss.
constexpr size_t kBoundsSlackBytes = size_t(1) << 16;
constexpr int64_t kBoundsSlackVertices = 1024;

__device__ __forceinline__ void bc_fail(int32_t* site_flag, int site) { atomicCAS(site_flag, 0, site); }

// v if it is a vertex ID in [0, n), else 0 (and the site is recorded).
__device__ __forceinline__ int32_t bc_vid(int32_t v, int64_t n, int32_t* site_flag, int site) {
  if (kBoundsCheck && (v < 0 || (int64_t)v >= n)) {
    bc_fail(site_flag, site);
    return 0;
  }
  return v;
}

// true if i is in [0, cap); otherwise records the site (the caller skips the access).
__device__ __forceinline__ bool bc_pos(int64_t i, int64_t cap, int32_t* site_flag, int site) {
  if (kBoundsCheck && (i < 0 || i >= cap)) {
    bc_fail(site_flag, site);
    return false;
  }
  return true;
}

// Clamps a row range to 0 <= s <= e <= nnz.
__device__ __forceinline__ void bc_row(int64_t& s, int64_t& e, int64_t nnz, int32_t* site_flag, int site) {
  if (kBoundsCheck && (s < 0 || s > e || e > nnz)) {
    bc_fail(site_flag, site);
    s = e = 0;
  }
}

enum BoundsSite {
  kBcTdFrontier = 1,  // top-down: frontier queue entry
  kBcTdRow,           // top-down: row offsets of a frontier vertex
  kBcTdColumn,        // top-down: neighbour ID
  kBcTdQueue,         // top-down: next-queue position
  kBcTdRecord,        // top-down: chunk record
  kBcConvert,         // queue <-> bitmap conversion
  kBcBuFirst,         // bottom-up: first neighbour
  kBcBuRow,           // bottom-up: row offsets
  kBcBuColumn,        // bottom-up: neighbour ID
  kBcBuDeferred,      // bottom-up: deferred-row list
  kBcOutput,          // output pass: parent or map entry
  kBcMsRow,           // batched: row offsets
  kBcMsColumn,        // batched: neighbour ID
  kBcMsRecord,        // batched: chunk record or deferred row
  kBcSiteCount
};

const char* bounds_site_name(int site);

// Sets a kernel's shared-memory carve-out to what min(per_sm, its occupancy)
// resident blocks of `threads` threads need, so the rest of the SM's on-chip
// memory serves as L1. Reverts to the default if the smaller carve-out would
// lower the kernel's occupancy. A hint only: results never depend on it.
template <class K>
void fit_carveout(K kernel, int threads, int per_sm) {
  int occ = 0, dev = 0, smem_sm = 0, reserve = 0;
  cudaFuncAttributes fa;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess || occ < 1 ||
      cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      smem_sm <= 0) {
    cudaGetLastError();
    return;
  }
  const int want = per_sm < occ ? per_sm : occ;
  const int64_t need = (int64_t)want * ((int64_t)fa.sharedSizeBytes + reserve);
  const int pct = (int)((need * 100 + smem_sm - 1) / smem_sm);
  int after = 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct < 100 ? pct : 100) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&after, kernel, threads, 0) != cudaSuccess || after < want)
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, -1);
  cudaGetLastError();
}

}  // namespace dobfs
