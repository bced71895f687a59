// LSD radix sort of 64-bit keys, used by the graph build (edge keys
// row<<b | col, and vertex keys by degree). Eight-bit digits; each pass is
// histogram -> exclusive scan -> stable scatter over P contiguous partitions
// (one CTA each), so a partition's keys of one digit land contiguously and in
// input order. Stability inside a CTA comes from ranking keys warp by warp
// with __match_any_sync: a warp owns a contiguous run of each tile, so the
// per-digit prefix over warps followed by the rank within the warp gives
// input order.
#include "common.cuh"
#include "sort.cuh"

namespace dobfs {

namespace {

constexpr int kRsThreads = 512;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 4;
constexpr int kRsTile = kRsWarps * kRsRounds * 32;  // 2048 keys per tile

__device__ __forceinline__ int64_t part_lo(int64_t n, int p, int P) {
  return (int64_t)(((unsigned __int128)n * (unsigned)p) / (unsigned)P);
}

__global__ void __launch_bounds__(kRsThreads) rs_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                      int shift, int P,
                                                      unsigned long long* __restrict__ hist) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int64_t lo = part_lo(n, blockIdx.x, P), hi = part_lo(n, blockIdx.x + 1, P);
  const unsigned lane = lane_id();
  // uniform trip count per warp so every lane takes part in match_any
  for (int64_t t = lo; t < hi; t += blockDim.x) {
    const int64_t i = t + threadIdx.x;
    const bool valid = i < hi;
    const unsigned d = valid ? (unsigned)((keys[i] >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (valid && (__ffs(peers) - 1) == (int)lane) atomicAdd(&h[d], (unsigned)__popc(peers));
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * P + blockIdx.x] = h[d];
}

// Exclusive scan of `len` counters in place, one CTA.
__global__ void __launch_bounds__(1024) rs_scan(unsigned long long* __restrict__ a, int64_t len) {
  __shared__ unsigned long long part[1024];
  const int64_t per = ceil_div(len, blockDim.x);
  const int64_t lo = per * threadIdx.x, hi = min(len, lo + per);
  unsigned long long s = 0;
  for (int64_t i = lo; i < hi; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const unsigned long long c = part[i];
      part[i] = run;
      run += c;
    }
  }
  __syncthreads();
  unsigned long long run = part[threadIdx.x];
  for (int64_t i = lo; i < hi; ++i) {
    const unsigned long long c = a[i];
    a[i] = run;
    run += c;
  }
}

__global__ void __launch_bounds__(kRsThreads) rs_scatter(const uint64_t* __restrict__ in,
                                                         uint64_t* __restrict__ out, int64_t n, int shift,
                                                         int P, const unsigned long long* __restrict__ hist) {
  __shared__ unsigned int wh[kRsWarps][256];
  __shared__ unsigned long long base[256];
  __shared__ unsigned int tot[256];
  for (int d = threadIdx.x; d < 256; d += blockDim.x) {
    base[d] = hist[(int64_t)d * P + blockIdx.x];
    for (int w = 0; w < kRsWarps; ++w) wh[w][d] = 0;
  }
  __syncthreads();
  const int64_t lo = part_lo(n, blockIdx.x, P), hi = part_lo(n, blockIdx.x + 1, P);
  const int w = threadIdx.x >> 5;
  const unsigned lane = lane_id();
  const unsigned lt = lanemask_lt();
  for (int64_t t = lo; t < hi; t += kRsTile) {
    uint64_t k[kRsRounds];
    unsigned dg[kRsRounds], rank[kRsRounds];
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
      const int64_t i = t + (int64_t)(w * kRsRounds + r) * 32 + lane;
      const bool valid = i < hi;
      k[r] = valid ? in[i] : 0ull;
      dg[r] = valid ? (unsigned)((k[r] >> shift) & 255u) : 256u;
    }
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
      const unsigned d = dg[r];
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const unsigned before = (d < 256u) ? wh[w][d] : 0u;
      rank[r] = before + (unsigned)__popc(peers & lt);
      __syncwarp();
      if (d < 256u && (__ffs(peers) - 1) == (int)lane) wh[w][d] = before + (unsigned)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
      unsigned run = 0;
#pragma unroll
      for (int ww = 0; ww < kRsWarps; ++ww) {
        const unsigned c = wh[ww][d];
        wh[ww][d] = run;
        run += c;
      }
      tot[d] = run;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
      const unsigned d = dg[r];
      if (d < 256u) out[base[d] + wh[w][d] + rank[r]] = k[r];
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
      base[d] += tot[d];
#pragma unroll
      for (int ww = 0; ww < kRsWarps; ++ww) wh[ww][d] = 0;
    }
    __syncthreads();
  }
}

}  // namespace

int radix_sort_u64(uint64_t* a, uint64_t* b, int64_t n, int nbits, cudaStream_t s, uint64_t** result) {
  *result = a;
  if (n <= 1 || nbits <= 0) return DOBFS_OK;
  const int P = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * 4, ceil_div(n, kRsTile)));
  DevBuf hist;
  DOBFS_TRY(hist.alloc(sizeof(unsigned long long) * 256 * (size_t)P, s));
  uint64_t* src = a;
  uint64_t* dst = b;
  for (int shift = 0; shift < nbits; shift += 8) {
    rs_hist<<<P, kRsThreads, 0, s>>>(src, n, shift, P, hist.as<unsigned long long>());
    rs_scan<<<1, 1024, 0, s>>>(hist.as<unsigned long long>(), (int64_t)256 * P);
    rs_scatter<<<P, kRsThreads, 0, s>>>(src, dst, n, shift, P, hist.as<unsigned long long>());
    DOBFS_CUDA_TRY(cudaGetLastError());
    std::swap(src, dst);
  }
  *result = src;
  // hist is freed on return; make sure the passes that read it are done
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  return DOBFS_OK;
}

}  // namespace dobfs
