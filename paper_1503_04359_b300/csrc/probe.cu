// Random-access rate of device memory: a measurement aid for the roofline of
// the BFS steps, whose accesses are mostly scattered reads and writes of 4
// to 16 bytes. DRAM serves each one as a whole 32-byte sector, and scattered
// sectors stream more slowly than a copy; this kernel gives the rate the
// memory system sustains for them, next to the copy bandwidth.
//
// Every thread makes `per_thread` accesses at positions drawn by a hash of
// its access number (no index array is read), eight at a time so that many
// accesses are in flight per thread; the grid fills every SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../dobfs_inputs/gen.h"
#include "common.cuh"

namespace dobfs {
namespace {

template <int WIDTH>
struct Slot;
template <>
struct Slot<4> { using T = uint32_t; };
template <>
struct Slot<8> { using T = unsigned long long; };
template <>
struct Slot<16> { using T = uint4; };

__device__ __forceinline__ uint32_t fold(uint32_t x) { return x; }
__device__ __forceinline__ uint32_t fold(unsigned long long x) { return (uint32_t)x ^ (uint32_t)(x >> 32); }
__device__ __forceinline__ uint32_t fold(uint4 x) { return x.x ^ x.y ^ x.z ^ x.w; }

template <int WIDTH>
__device__ __forceinline__ typename Slot<WIDTH>::T make_slot(uint32_t v) {
  if constexpr (WIDTH == 4) return v;
  else if constexpr (WIDTH == 8) return (unsigned long long)v;
  else return make_uint4(v, v, v, v);
}

template <int WIDTH, bool WRITE>
__global__ void __launch_bounds__(256) k_random_access(typename Slot<WIDTH>::T* arr, uint64_t slot_mask,
                                                      uint64_t seed, int64_t per_thread, uint32_t* sink) {
  constexpr int kInFlight = 8;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (int64_t i = 0; i < per_thread; i += kInFlight) {
    uint64_t pos[kInFlight];
#pragma unroll
    for (int k = 0; k < kInFlight; ++k) pos[k] = gen_mix64(seed ^ (tid * (uint64_t)per_thread + (uint64_t)(i + k))) & slot_mask;
    if constexpr (WRITE) {
#pragma unroll
      for (int k = 0; k < kInFlight; ++k) arr[pos[k]] = make_slot<WIDTH>((uint32_t)(i + k));
    } else {
      typename Slot<WIDTH>::T x[kInFlight];
#pragma unroll
      for (int k = 0; k < kInFlight; ++k) x[k] = arr[pos[k]];
#pragma unroll
      for (int k = 0; k < kInFlight; ++k) acc ^= fold(x[k]);
    }
  }
  if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps the loads; practically never taken
}

template <int WIDTH, bool WRITE>
int launch_probe(void* arr, int64_t array_bytes, int64_t accesses, uint32_t* sink, float* ms_out,
                 int64_t* made_out) {
  auto kern = k_random_access<WIDTH, WRITE>;
  int per_sm = 0;
  DOBFS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0));
  const int64_t threads = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1) * 256;
  const int64_t per_thread = (int64_t)ceil_div(ceil_div(accesses, threads), 8) * 8;
  const uint64_t mask = (uint64_t)(array_bytes / WIDTH) - 1;
  const int grid = (int)(threads / 256);
  cudaEvent_t e0, e1;
  DOBFS_CUDA_TRY(cudaEventCreate(&e0));
  DOBFS_CUDA_TRY(cudaEventCreate(&e1));
  using T = typename Slot<WIDTH>::T;
  kern<<<grid, 256>>>(static_cast<T*>(arr), mask, 1ull, per_thread, sink);  // warm-up
  cudaEventRecord(e0);
  kern<<<grid, 256>>>(static_cast<T*>(arr), mask, 2ull, per_thread, sink);
  cudaEventRecord(e1);
  const cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  DOBFS_CUDA_TRY(err);
  DOBFS_CUDA_TRY(cudaGetLastError());
  *ms_out = ms;
  *made_out = per_thread * threads;  // the request rounded up to whole rounds of the grid
  return DOBFS_OK;
}

}  // namespace
}  // namespace dobfs

using namespace dobfs;

extern "C" int dobfs_debug_random_access(int64_t array_bytes, int64_t accesses, int32_t width, int32_t write,
                                         float* ms_out, int64_t* made_out) {
  clear_error();
  if (!ms_out || !made_out) return set_error(DOBFS_ERR_INVALID, "output pointers are NULL");
  if (array_bytes < (int64_t(1) << 20) || (array_bytes & (array_bytes - 1)) != 0 || accesses < 1 ||
      !(width == 4 || width == 8 || width == 16) || (write != 0 && write != 1))
    return set_error(DOBFS_ERR_INVALID,
                     "bad probe: array_bytes %lld (a power of two >= 1 MB), accesses %lld, width %d (4, 8, 16), "
                     "write %d",
                     (long long)array_bytes, (long long)accesses, width, write);
  DevBuf arr, sink;
  DOBFS_TRY(arr.alloc((size_t)array_bytes, nullptr));
  DOBFS_TRY(sink.alloc(sizeof(uint32_t), nullptr));
  DOBFS_CUDA_TRY(cudaMemsetAsync(arr.ptr, 0, (size_t)array_bytes, nullptr));
  uint32_t* s = sink.as<uint32_t>();
  int rc;
  if (width == 4) rc = write ? launch_probe<4, true>(arr.ptr, array_bytes, accesses, s, ms_out, made_out)
                             : launch_probe<4, false>(arr.ptr, array_bytes, accesses, s, ms_out, made_out);
  else if (width == 8) rc = write ? launch_probe<8, true>(arr.ptr, array_bytes, accesses, s, ms_out, made_out)
                                  : launch_probe<8, false>(arr.ptr, array_bytes, accesses, s, ms_out, made_out);
  else rc = write ? launch_probe<16, true>(arr.ptr, array_bytes, accesses, s, ms_out, made_out)
                  : launch_probe<16, false>(arr.ptr, array_bytes, accesses, s, ms_out, made_out);
  cudaDeviceSynchronize();
  return rc;
}
