// Graph construction on the device.
//
// Every input (pairs, CSR arrays, or the R-MAT / Chung-Lu generators of
// dobfs_inputs/gen.h) is turned into 64-bit edge keys row<<b | col (b bits
// per vertex ID), with self-loops mapped to a sentinel that sorts last. One
// LSD radix sort over 2b bits orders the keys by (row, col); a partitioned
// compaction drops duplicates and writes the columns and row offsets. The
// CSR stores each undirected edge as two directed entries (Sec. 4,
// "Methodology").
//
// Degree-sorted reindexing (Sec. 3.4): vertices are renumbered by decreasing
// degree (ties by increasing original ID) and every key is relabelled and
// sorted again, so rows come in new-ID order and each row lists its
// neighbours by increasing new ID, i.e. by decreasing degree — the highest-
// degree neighbour first, which shortens bottom-up scans.
#include <algorithm>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include "../../dobfs_inputs/gen.h"
#include "common.cuh"
#include "graph.cuh"
#include "sort.cuh"

namespace dobfs {

namespace {

constexpr int kThreads = 256;
constexpr uint64_t kHubDegree = 4096;   // degrees from here on keep their exact order
constexpr uint64_t kQuantClasses = 64;  // above the largest quantised class (43)

__device__ __forceinline__ int64_t part_lo(int64_t n, int p, int P) {
  return (int64_t)(((unsigned __int128)n * (unsigned)p) / (unsigned)P);
}

__device__ __forceinline__ uint64_t edge_key(uint32_t u, uint32_t v, int b) {
  return u == v ? kSentinelKey : (((uint64_t)u << b) | (uint64_t)v);
}

__global__ void k_keys_pairs(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                             int64_t n, int b, uint64_t* __restrict__ keys, int* __restrict__ err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = src[i], v = dst[i];
    if (u < 0 || v < 0 || u >= n || v >= n) {
      atomicExch(err, 1);
      keys[2 * i] = kSentinelKey;
      keys[2 * i + 1] = kSentinelKey;
      continue;
    }
    keys[2 * i] = edge_key((uint32_t)u, (uint32_t)v, b);
    keys[2 * i + 1] = edge_key((uint32_t)v, (uint32_t)u, b);
  }
}

__global__ void k_keys_rmat(int64_t m, int scale, uint32_t ta, uint32_t tab, uint32_t tabc, uint64_t kp,
                            uint64_t kq, int b, uint64_t* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t u, v;
    gen_rmat_pair((uint64_t)i, scale, ta, tab, tabc, kp, kq, &u, &v);
    keys[2 * i] = edge_key(u, v, b);
    keys[2 * i + 1] = edge_key(v, u, b);
  }
}

__global__ void k_keys_chunglu(const uint64_t* __restrict__ cdf, uint32_t n, int64_t m, uint64_t kp,
                               uint64_t kq, int b, uint64_t* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t u, v;
    gen_chunglu_pair((uint64_t)i, cdf, n, kp, kq, &u, &v);
    keys[2 * i] = edge_key(u, v, b);
    keys[2 * i + 1] = edge_key(v, u, b);
  }
}

// One warp per row; with `sym` the reverse entry goes to keys[nnz + j].
template <class OffT>
__global__ void k_keys_csr(const OffT* __restrict__ off, const int32_t* __restrict__ cols, int64_t n,
                           int64_t nnz, int b, int sym, uint64_t* __restrict__ keys, int* __restrict__ err) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    const int64_t s = (int64_t)off[u], e = (int64_t)off[u + 1];
    if (s < 0 || e < s || e > nnz) {
      if (lane_id() == 0) atomicExch(err, 2);
      continue;
    }
    for (int64_t j = s + lane_id(); j < e; j += 32) {
      const int32_t v = cols[j];
      if (v < 0 || v >= n) {
        atomicExch(err, 1);
        keys[j] = kSentinelKey;
        if (sym) keys[nnz + j] = kSentinelKey;
        continue;
      }
      keys[j] = edge_key((uint32_t)u, (uint32_t)v, b);
      if (sym) keys[nnz + j] = edge_key((uint32_t)v, (uint32_t)u, b);
    }
  }
}

__device__ __forceinline__ bool key_kept(const uint64_t* __restrict__ keys, int64_t i, uint64_t* k_out,
                                         uint64_t* kprev_out) {
  const uint64_t k = keys[i];
  *k_out = k;
  if (k == kSentinelKey) return false;
  if (i == 0) return true;
  const uint64_t kp = keys[i - 1];
  *kprev_out = kp;
  return k != kp;
}

// Kept (non-sentinel, non-duplicate) keys per partition.
__global__ void __launch_bounds__(kThreads) k_count_kept(const uint64_t* __restrict__ keys, int64_t m, int P,
                                                         unsigned long long* __restrict__ counts) {
  __shared__ unsigned long long sh[kThreads / 32];
  const int64_t lo = part_lo(m, blockIdx.x, P), hi = part_lo(m, blockIdx.x + 1, P);
  unsigned long long c = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    uint64_t k, kp;
    c += key_kept(keys, i, &k, &kp) ? 1 : 0;
  }
  c = block_sum_u64(c, sh);
  if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// Exclusive scan of P counts in place; total into counts[P].
__global__ void k_scan_small(unsigned long long* counts, int P) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned long long run = 0;
  for (int i = 0; i < P; ++i) {
    const unsigned long long c = counts[i];
    counts[i] = run;
    run += c;
  }
  counts[P] = run;
}

// Writes the kept keys' columns (if cols) and the row offsets up to the last
// non-empty row. Each such offset is written exactly once: by the first kept
// key of the row, which also fills the offsets of the empty rows before it.
// k_fill_tail writes the offsets after the last non-empty row.
template <class OffT>
__global__ void __launch_bounds__(kThreads) k_extract(const uint64_t* __restrict__ keys, int64_t m, int b, int P,
                                                      const unsigned long long* __restrict__ base,
                                                      OffT* __restrict__ off, int32_t* __restrict__ cols,
                                                      int64_t n) {
  __shared__ unsigned warp_cnt[kThreads / 32];
  __shared__ unsigned long long running;
  const int64_t lo = part_lo(m, blockIdx.x, P), hi = part_lo(m, blockIdx.x + 1, P);
  if (threadIdx.x == 0) running = base[blockIdx.x];
  __syncthreads();
  const uint64_t cmask = (1ull << b) - 1ull;
  const int w = threadIdx.x >> 5;
  for (int64_t t = lo; t < hi; t += blockDim.x) {
    const int64_t i = t + threadIdx.x;
    uint64_t k = 0, kp = 0;
    const bool kept = (i < hi) && key_kept(keys, i, &k, &kp);
    const unsigned bal = __ballot_sync(0xffffffffu, kept);
    if (lane_id() == 0) warp_cnt[w] = (unsigned)__popc(bal);
    __syncthreads();
    unsigned wpre = 0, tot = 0;
    for (int j = 0; j < kThreads / 32; ++j) {
      wpre += (j < w) ? warp_cnt[j] : 0u;
      tot += warp_cnt[j];
    }
    const unsigned long long pos = running + wpre + (unsigned)__popc(bal & lanemask_lt());
    if (kept) {
      if (cols) cols[pos] = (int32_t)(k & cmask);
      const int64_t r = (int64_t)(k >> b);
      const int64_t rp = (i == 0) ? -1 : (int64_t)(kp >> b);
      for (int64_t rr = rp + 1; rr <= r; ++rr) off[rr] = (OffT)pos;
    }
    __syncthreads();
    if (threadIdx.x == 0) running += tot;
    __syncthreads();
  }
}

// off[r] = total for every row after the last non-empty one. The last kept
// key is the one before the first sentinel of the sorted array.
template <class OffT>
__global__ void k_fill_tail(const uint64_t* __restrict__ keys, int64_t m, int b, OffT* __restrict__ off, int64_t n,
                            int64_t total) {
  int64_t lo = 0, hi = m;  // first index holding the sentinel
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (keys[mid] == kSentinelKey) hi = mid; else lo = mid + 1;
  }
  if (lo == 0) return;  // no kept key: offsets stay 0
  const int64_t r_last = (int64_t)(keys[lo - 1] >> b);
  for (int64_t r = r_last + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= n;
       r += (int64_t)gridDim.x * blockDim.x)
    off[r] = (OffT)total;
}

// Symmetry check on sorted keys: every kept key's reverse must be present.
__global__ void k_check_sym(const uint64_t* __restrict__ keys, int64_t m, int b, int* __restrict__ err) {
  const uint64_t cmask = (1ull << b) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k, kp;
    if (!key_kept(keys, i, &k, &kp)) continue;
    const uint64_t want = ((k & cmask) << b) | (k >> b);
    int64_t lo = 0, hi = m;
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (keys[mid] < want) lo = mid + 1; else hi = mid;
    }
    if (lo >= m || keys[lo] != want) atomicExch(err, 3);
  }
}

// Bitmap of degree-0 vertices (and of the padding bits >= n), the count of
// vertices with an edge, and the maximum degree. One thread per vertex; a
// warp covers one bitmap word.
template <class OffT>
__global__ void k_deg_stats(const OffT* __restrict__ off, int64_t n, int64_t words, uint32_t* __restrict__ iso,
                            unsigned long long* __restrict__ stats) {
  // stats: [0] vertices with an edge, [1] max degree, [2 + k] vertices with
  // floor(log2(degree)) == k, [34 + d] vertices of degree d (d < kSmallDeg)
  __shared__ unsigned long long sh[kThreads / 32];
  __shared__ unsigned int s_hist[32];
  __shared__ unsigned int s_small[kSmallDeg];
  if (threadIdx.x < 32) s_hist[threadIdx.x] = 0u;
  if (threadIdx.x < kSmallDeg) s_small[threadIdx.x] = 0u;
  __syncthreads();
  unsigned long long nonzero = 0, mx = 0;
  const int64_t total = words * 32;
  for (int64_t v0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; v0 < total;
       v0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = v0 + lane_id();
    bool isolated = true;
    if (v < n) {
      const int64_t d = (int64_t)off[v + 1] - (int64_t)off[v];
      isolated = (d == 0);
      nonzero += isolated ? 0 : 1;
      mx = max(mx, (unsigned long long)d);
      if (!isolated) atomicAdd(&s_hist[63 - __clzll((unsigned long long)d)], 1u);
      if (d < kSmallDeg) atomicAdd(&s_small[d], 1u);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, isolated);
    if (lane_id() == 0) iso[v0 >> 5] = bal;
  }
  __syncthreads();
  if (threadIdx.x < 32 && s_hist[threadIdx.x]) atomicAdd(&stats[2 + threadIdx.x], (unsigned long long)s_hist[threadIdx.x]);
  if (threadIdx.x < kSmallDeg && s_small[threadIdx.x])
    atomicAdd(&stats[34 + threadIdx.x], (unsigned long long)s_small[threadIdx.x]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if (lane_id() == 0) atomicMax(&stats[1], mx);
  nonzero = block_sum_u64(nonzero, sh);
  if (threadIdx.x == 0) atomicAdd(&stats[0], nonzero);
}

// Degree class used by the renumbering. Exact order (DOBFS_GRAPH_REINDEX_EXACT):
// the degree itself. Class order (DOBFS_GRAPH_REINDEX): degrees below 8 are
// their own class, degrees in [8, 4096) are cut into four classes per
// octave (the two bits below the leading one), and degrees of 4096 and more
// (the hubs) keep their exact order above every quantised class. Both are
// non-decreasing in the degree, so the renumbering stays by decreasing
// degree up to ties inside a class, which are broken by original ID.
__device__ __forceinline__ uint64_t degree_class(uint64_t d, bool exact) {
  if (exact || d >= kHubDegree) return exact ? d : kQuantClasses + d;
  if (d < 8) return d;
  const int e = 63 - __clzll((long long)d);  // floor(log2 d) >= 3
  return 8 + 4 * (uint64_t)(e - 3) + ((d >> (e - 2)) & 3ull);
}

// Vertex keys for the renumbering: (cmax - class(degree)) << b | id, so an
// ascending sort gives decreasing class, ties by increasing original ID.
__global__ void k_vertex_keys(const int64_t* __restrict__ off, int64_t n, int b, int cls_bits, int exact,
                              uint64_t* __restrict__ keys) {
  const uint64_t cmax = (1ull << cls_bits) - 1ull;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t d = (uint64_t)(off[u + 1] - off[u]);
    keys[u] = ((cmax - degree_class(d, exact != 0)) << b) | (uint64_t)u;
  }
}

__global__ void k_maps(const uint64_t* __restrict__ sorted, int64_t n, int b, int32_t* __restrict__ new2orig,
                       int32_t* __restrict__ orig2new) {
  const uint64_t mask = (1ull << b) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = (int32_t)(sorted[i] & mask);
    new2orig[i] = o;
    orig2new[o] = (int32_t)i;
  }
}

// Relabels the kept keys of a sorted array into `out`; dropped keys become
// the sentinel.
__global__ void k_relabel(const uint64_t* __restrict__ keys, int64_t m, int b, const int32_t* __restrict__ o2n,
                          uint64_t* __restrict__ out) {
  const uint64_t mask = (1ull << b) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k, kp;
    if (!key_kept(keys, i, &k, &kp)) {
      out[i] = kSentinelKey;
      continue;
    }
    const uint32_t u = (uint32_t)o2n[k >> b], v = (uint32_t)o2n[k & mask];
    out[i] = ((uint64_t)u << b) | (uint64_t)v;
  }
}

__global__ void k_widen(const int32_t* __restrict__ a, int64_t n, int64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i];
}

__global__ void k_iota(int32_t* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)i;
}

template <class OffT>
__global__ void k_degrees(const OffT* __restrict__ off, const int32_t* __restrict__ o2n, int64_t n,
                          int32_t* __restrict__ deg) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = o2n ? o2n[o] : o;
    deg[o] = (int32_t)((int64_t)off[v + 1] - (int64_t)off[v]);
  }
}

int grid_for(int64_t work, int threads = kThreads) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, threads), (int64_t)sm_count() * 16));
}

// Counts kept keys per partition and scans: base[P] exclusive, base[P] = total.
int kept_bases(const uint64_t* keys, int64_t m, int P, DevBuf& base, cudaStream_t s, int64_t* total) {
  DOBFS_TRY(base.alloc(sizeof(unsigned long long) * (P + 1), s));
  k_count_kept<<<P, kThreads, 0, s>>>(keys, m, P, base.as<unsigned long long>());
  k_scan_small<<<1, 1, 0, s>>>(base.as<unsigned long long>(), P);
  DOBFS_CUDA_TRY(cudaGetLastError());
  unsigned long long t = 0;
  DOBFS_CUDA_TRY(cudaMemcpyAsync(&t, base.as<unsigned long long>() + P, sizeof(t), cudaMemcpyDeviceToHost, s));
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  *total = (int64_t)t;
  return DOBFS_OK;
}

template <class OffT>
int extract(const uint64_t* keys, int64_t m, int b, int64_t n, OffT* off, int32_t* cols, cudaStream_t s,
            int64_t* nnz_out) {
  const int P = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * 4, ceil_div(m, 4096)));
  DevBuf base;
  int64_t total = 0;
  DOBFS_TRY(kept_bases(keys, m, P, base, s, &total));
  DOBFS_CUDA_TRY(cudaMemsetAsync(off, 0, sizeof(OffT) * (size_t)(n + 1), s));
  if (m > 0) {
    k_extract<OffT><<<P, kThreads, 0, s>>>(keys, m, b, P, base.as<unsigned long long>(), off, cols, n);
    k_fill_tail<OffT><<<grid_for(n + 1), kThreads, 0, s>>>(keys, m, b, off, n, total);
  }
  DOBFS_CUDA_TRY(cudaGetLastError());
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  *nnz_out = total;
  return DOBFS_OK;
}

template <class OffT>
int finish_stats(dobfs_graph* g, cudaStream_t s) {
  g->words = ceil_div(g->n, 32);
  DOBFS_TRY(g->isolated.alloc(sizeof(uint32_t) * (size_t)g->words, s));
  DevBuf st;
  constexpr int kStats = 34 + kSmallDeg;
  DOBFS_TRY(st.alloc(sizeof(unsigned long long) * kStats, s));
  DOBFS_CUDA_TRY(cudaMemsetAsync(st.ptr, 0, sizeof(unsigned long long) * kStats, s));
  k_deg_stats<OffT><<<grid_for(g->words * 32), kThreads, 0, s>>>(g->off.as<OffT>(), g->n, g->words,
                                                                  g->isolated.as<uint32_t>(),
                                                                  st.as<unsigned long long>());
  DOBFS_CUDA_TRY(cudaGetLastError());
  unsigned long long h[kStats];
  DOBFS_CUDA_TRY(cudaMemcpyAsync(h, st.ptr, sizeof(h), cudaMemcpyDeviceToHost, s));
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  g->n_nonisolated = (int64_t)h[0];
  g->max_degree = (int64_t)h[1];
  // vertices of degree >= 2^k; with the degree-sorted renumbering they are
  // the first deg_ge[k] vertex IDs (every power of two is a class boundary)
  int64_t acc = 0;
  for (int k = 32; k >= 0; --k) {
    if (k < 32) acc += (int64_t)h[2 + k];
    g->deg_ge[k] = acc;
  }
  // Renumbered graphs: each degree d below kSmallDeg is a class of its own,
  // so its vertices are consecutive and their rows (d entries each) too:
  // row_start(v) = base[d] + (v - first[d]) * d, with first[d] the number
  // of vertices of degree above d and base[d] its row offset.
  memset(g->small_tab, 0, sizeof(g->small_tab));
  g->small_deg = 0;
  if (g->reindexed) {
    int64_t above = g->n_nonisolated;  // vertices of degree > d, for d = 0
    for (int d = 1; d < kSmallDeg; ++d) {
      above -= (int64_t)h[34 + d];
      g->small_tab[kSmallDeg + d] = above;
      OffT base = 0;
      DOBFS_CUDA_TRY(cudaMemcpyAsync(&base, g->off.as<OffT>() + above, sizeof(OffT), cudaMemcpyDeviceToHost, s));
      DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
      g->small_tab[d] = (int64_t)base;
    }
    g->small_deg = kSmallDeg;
  }
  return DOBFS_OK;
}

// ---------------------------------------------------------------- chunked R-MAT build
// The one-shot build holds 16 bytes of key scratch per directed entry (two
// 64-bit key buffers), 275 GB at scale 29. The chunked build never holds
// more than one chunk of keys: the counter-based edge stream is regenerated
// for every chunk of source rows, and a chunk's keys are sorted,
// de-duplicated and written straight into the final CSR. Two passes: the
// first (original IDs) finds each vertex's degree and raw entry count, the
// renumbering is computed from the degrees, the second writes the columns
// in the final IDs. The result is identical to the one-shot build's.

constexpr int kHistBuckets = 4096;

// Raw directed entries (self-loops dropped) per bucket of source IDs.
__global__ void __launch_bounds__(kThreads) k_rmat_src_hist(int64_t m, int scale, uint32_t ta, uint32_t tab,
                                                            uint32_t tabc, uint64_t kp, uint64_t kq, int shift,
                                                            unsigned long long* __restrict__ hist) {
  __shared__ unsigned int h[kHistBuckets];
  for (int i = threadIdx.x; i < kHistBuckets; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t u, v;
    gen_rmat_pair((uint64_t)i, scale, ta, tab, tabc, kp, kq, &u, &v);
    if (u == v) continue;
    atomicAdd(&h[u >> shift], 1u);
    atomicAdd(&h[v >> shift], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kHistBuckets; i += blockDim.x)
    if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

// Keys ((src - lo) << b | dst) of the directed entries whose source, after
// the optional renumbering `map`, lies in [lo, hi); positions from one
// warp-aggregated atomic per direction. Entries past `cap` are counted, not
// written (the caller sizes chunks so that this does not happen).
__global__ void __launch_bounds__(kThreads) k_keys_rmat_range(int64_t m, int scale, uint32_t ta, uint32_t tab,
                                                              uint32_t tabc, uint64_t kp, uint64_t kq,
                                                              const int32_t* __restrict__ map, int64_t lo,
                                                              int64_t hi, int b, int64_t cap,
                                                              uint64_t* __restrict__ keys,
                                                              unsigned long long* __restrict__ count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; i0 < m; i0 += stride) {
    const int64_t i = i0 + lane_id();
    uint32_t u = 0, v = 0;
    bool ok = i < m;
    if (ok) {
      gen_rmat_pair((uint64_t)i, scale, ta, tab, tabc, kp, kq, &u, &v);
      ok = (u != v);
      if (ok && map) {
        u = (uint32_t)__ldg(map + u);
        v = (uint32_t)__ldg(map + v);
      }
    }
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const uint32_t src = dir ? v : u, dst = dir ? u : v;
      const bool in = ok && (int64_t)src >= lo && (int64_t)src < hi;
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      if (!bal) continue;
      unsigned long long base = 0;
      if (lane_id() == 0) base = atomicAdd(count, (unsigned long long)__popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      const unsigned long long pos = base + (unsigned)__popc(bal & lanemask_lt());
      if (in && (int64_t)pos < cap) keys[pos] = ((uint64_t)((int64_t)src - lo) << b) | (uint64_t)dst;
    }
  }
}

// raw[r] = first position of row r in the sorted chunk keys (r in [0, rows]).
__global__ void k_row_starts(const uint64_t* __restrict__ keys, int64_t m, int b, int64_t rows,
                             int64_t* __restrict__ raw) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= rows; r += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t want = (uint64_t)r << b;
    int64_t a = 0, z = m;
    while (a < z) {
      const int64_t mid = a + ((z - a) >> 1);
      if (keys[mid] < want) a = mid + 1; else z = mid;
    }
    raw[r] = a;
  }
}

// Degree (entries kept) and raw entry count of the chunk's rows.
__global__ void k_chunk_degrees(const int64_t* __restrict__ off, const int64_t* __restrict__ raw, int64_t rows,
                                int64_t lo, int32_t* __restrict__ deg, int32_t* __restrict__ rawdeg) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    deg[lo + r] = (int32_t)(off[r + 1] - off[r]);
    rawdeg[lo + r] = (int32_t)(raw[r + 1] - raw[r]);
  }
}

__global__ void k_vertex_keys_deg(const int32_t* __restrict__ deg, int64_t n, int b, int cls_bits, int exact,
                                  uint64_t* __restrict__ keys) {
  const uint64_t cmax = (1ull << cls_bits) - 1ull;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    keys[u] = ((cmax - degree_class((uint64_t)deg[u], exact != 0)) << b) | (uint64_t)u;
}

// In final order: d[i] = degree, r[i] = raw count of vertex n2o[i] (or i).
__global__ void k_gather_counts(const int32_t* __restrict__ n2o, const int32_t* __restrict__ deg,
                                const int32_t* __restrict__ rawdeg, int64_t n, int64_t* __restrict__ d,
                                int64_t* __restrict__ r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = n2o ? n2o[i] : i;
    d[i] = deg[o];
    r[i] = rawdeg[o];
  }
}

// Exclusive scan of x[0, n) in place with x[n] = total: tile sums, a scan of
// the tile sums by one block, then each tile's scan plus its base.
constexpr int kScanTile = kThreads * 16;

__global__ void __launch_bounds__(kThreads) k_scan_tiles(const int64_t* __restrict__ x, int64_t n,
                                                         unsigned long long* __restrict__ tsum) {
  __shared__ unsigned long long sh[kThreads / 32];
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
  unsigned long long acc = 0;
  for (int64_t i = t0 + threadIdx.x; i < min(n, t0 + kScanTile); i += blockDim.x) acc += (unsigned long long)x[i];
  acc = block_sum_u64(acc, sh);
  if (threadIdx.x == 0) tsum[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(1024) k_scan_tile_sums(unsigned long long* __restrict__ tsum, int64_t tiles) {
  __shared__ unsigned long long part[1024];
  const int64_t per = ceil_div(tiles, (int64_t)blockDim.x);
  const int64_t a = threadIdx.x * per, z = min(tiles, a + per);
  unsigned long long s = 0;
  for (int64_t i = a; i < z; ++i) s += tsum[i];
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
  for (int64_t i = a; i < z; ++i) {
    const unsigned long long c = tsum[i];
    tsum[i] = run;
    run += c;
  }
}

template <class OutT>
__global__ void __launch_bounds__(kThreads) k_scan_apply(const int64_t* __restrict__ x, int64_t n,
                                                         const unsigned long long* __restrict__ tsum,
                                                         OutT* __restrict__ out) {
  __shared__ unsigned long long s_part[kThreads];
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
  const int64_t t1 = min(n, t0 + kScanTile);
  // each thread scans a contiguous run of 16, then a block scan of the runs
  const int64_t a = t0 + (int64_t)threadIdx.x * 16, z = min(t1, a + 16);
  unsigned long long local = 0;
  for (int64_t i = a; i < z; ++i) local += (unsigned long long)x[i];
  s_part[threadIdx.x] = local;
  __syncthreads();
  for (int o = 1; o < kThreads; o <<= 1) {
    const unsigned long long y = (threadIdx.x >= (unsigned)o) ? s_part[threadIdx.x - o] : 0ull;
    __syncthreads();
    s_part[threadIdx.x] += y;
    __syncthreads();
  }
  unsigned long long run = tsum[blockIdx.x] + s_part[threadIdx.x] - local;
  for (int64_t i = a; i < z; ++i) {
    const unsigned long long c = (unsigned long long)x[i];
    out[i] = (OutT)run;
    run += c;
  }
  if (z == n && a < z) out[n] = (OutT)run;  // the thread holding the last element writes the total
}

// out[0, n] = exclusive scan of x[0, n), out[n] = total. Returns the total.
template <class OutT>
int exclusive_scan(const int64_t* x, int64_t n, OutT* out, cudaStream_t s, int64_t* total) {
  const int64_t tiles = std::max<int64_t>(1, ceil_div(n, (int64_t)kScanTile));
  DevBuf tsum;
  DOBFS_TRY(tsum.alloc(sizeof(unsigned long long) * (size_t)tiles, s));
  k_scan_tiles<<<(unsigned)tiles, kThreads, 0, s>>>(x, n, tsum.as<unsigned long long>());
  k_scan_tile_sums<<<1, 1024, 0, s>>>(tsum.as<unsigned long long>(), tiles);
  k_scan_apply<OutT><<<(unsigned)tiles, kThreads, 0, s>>>(x, n, tsum.as<unsigned long long>(), out);
  DOBFS_CUDA_TRY(cudaGetLastError());
  OutT t = 0;
  DOBFS_CUDA_TRY(cudaMemcpyAsync(&t, out + n, sizeof(OutT), cudaMemcpyDeviceToHost, s));
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  *total = (int64_t)t;
  return DOBFS_OK;
}

struct RmatGen {
  int scale;
  int64_t m;  // pairs
  uint32_t ta, tab, tabc;
  uint64_t kp, kq;
};

// One chunk: keys of sources [lo, hi) (after `map`), sorted. *m_out = count.
int chunk_keys(const RmatGen& G, const int32_t* map, int64_t lo, int64_t hi, int b, DevBuf& ka, DevBuf& kb,
               int64_t cap, cudaStream_t s, uint64_t** sorted, int64_t* m_out) {
  DevBuf cnt;
  DOBFS_TRY(cnt.alloc(sizeof(unsigned long long), s));
  DOBFS_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, sizeof(unsigned long long), s));
  k_keys_rmat_range<<<grid_for(G.m), kThreads, 0, s>>>(G.m, G.scale, G.ta, G.tab, G.tabc, G.kp, G.kq, map, lo, hi,
                                                      b, cap, ka.as<uint64_t>(), cnt.as<unsigned long long>());
  DOBFS_CUDA_TRY(cudaGetLastError());
  unsigned long long c = 0;
  DOBFS_CUDA_TRY(cudaMemcpyAsync(&c, cnt.ptr, sizeof(c), cudaMemcpyDeviceToHost, s));
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  if ((int64_t)c > cap) return set_error(DOBFS_ERR_OOM, "internal: chunk of %llu keys exceeds %lld", c, (long long)cap);
  const int rbits = std::max(1, bits_for(std::max<int64_t>(hi - lo, 2)));
  DOBFS_TRY(radix_sort_u64(ka.as<uint64_t>(), kb.as<uint64_t>(), (int64_t)c, rbits + b, s, sorted));
  *m_out = (int64_t)c;
  return DOBFS_OK;
}

int read_i64(const int64_t* p, cudaStream_t s, int64_t* v) {
  DOBFS_CUDA_TRY(cudaMemcpyAsync(v, p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  return DOBFS_OK;
}

template <class OffT>
int chunked_fill(dobfs_graph* g, const RmatGen& G, const int64_t* rawpre, DevBuf& ka, DevBuf& kb, int64_t cap,
                 cudaStream_t s) {
  const int b = g->bits;
  const int64_t n = g->n;
  const int32_t* map = g->reindexed ? g->orig2new.as<int32_t>() : nullptr;
  OffT* off = g->off.as<OffT>();
  int64_t lo = 0;
  while (lo < n) {
    // the longest run of rows from lo whose raw entries fit in the chunk
    int64_t base = 0;
    DOBFS_TRY(read_i64(rawpre + lo, s, &base));
    int64_t a = lo + 1, z = n;  // largest hi in [lo+1, n] with rawpre[hi] - base <= cap
    int64_t v = 0;
    DOBFS_TRY(read_i64(rawpre + a, s, &v));
    if (v - base > cap) return set_error(DOBFS_ERR_OOM, "a row exceeds the build chunk");
    while (a < z) {
      const int64_t mid = a + ((z - a + 1) >> 1);
      DOBFS_TRY(read_i64(rawpre + mid, s, &v));
      if (v - base <= cap) a = mid; else z = mid - 1;
    }
    const int64_t hi = a;
    uint64_t* sorted = nullptr;
    int64_t mc = 0;
    DOBFS_TRY(chunk_keys(G, map, lo, hi, b, ka, kb, cap, s, &sorted, &mc));
    int64_t o_lo = 0;
    OffT t = 0;
    DOBFS_CUDA_TRY(cudaMemcpyAsync(&t, off + lo, sizeof(OffT), cudaMemcpyDeviceToHost, s));
    DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
    o_lo = (int64_t)t;
    DevBuf offc;
    DOBFS_TRY(offc.alloc(sizeof(int64_t) * (size_t)(hi - lo + 1), s));
    int64_t kept = 0;
    DOBFS_TRY(extract<int64_t>(sorted, mc, b, hi - lo, offc.as<int64_t>(), g->cols.as<int32_t>() + o_lo, s, &kept));
    DOBFS_CUDA_TRY(cudaMemcpyAsync(&t, off + hi, sizeof(OffT), cudaMemcpyDeviceToHost, s));
    DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
    if ((int64_t)t - o_lo != kept) return set_error(DOBFS_ERR_CUDA, "internal: chunk entry count changed between passes");
    lo = hi;
  }
  return DOBFS_OK;
}

int build_rmat_chunked(dobfs_graph* g, const RmatGen& G, uint32_t flags, int64_t cap, cudaStream_t s) {
  const int b = g->bits;
  const int64_t n = g->n;
  DevBuf ka, kb;
  DOBFS_TRY(ka.alloc(sizeof(uint64_t) * (size_t)cap, s));
  DOBFS_TRY(kb.alloc(sizeof(uint64_t) * (size_t)cap, s));
  // pass 1 (original IDs): plan chunks on a histogram of the sources
  const int shift = std::max(0, b - 12);
  std::vector<unsigned long long> hist(kHistBuckets, 0ull);
  {
    DevBuf dh;
    DOBFS_TRY(dh.alloc(sizeof(unsigned long long) * kHistBuckets, s));
    DOBFS_CUDA_TRY(cudaMemsetAsync(dh.ptr, 0, sizeof(unsigned long long) * kHistBuckets, s));
    k_rmat_src_hist<<<grid_for(G.m), kThreads, 0, s>>>(G.m, G.scale, G.ta, G.tab, G.tabc, G.kp, G.kq, shift,
                                                      dh.as<unsigned long long>());
    DOBFS_CUDA_TRY(cudaGetLastError());
    DOBFS_CUDA_TRY(cudaMemcpyAsync(hist.data(), dh.ptr, sizeof(unsigned long long) * kHistBuckets,
                                   cudaMemcpyDeviceToHost, s));
    DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  DevBuf deg, rawdeg;
  DOBFS_TRY(deg.alloc(sizeof(int32_t) * (size_t)n, s));
  DOBFS_TRY(rawdeg.alloc(sizeof(int32_t) * (size_t)n, s));
  {
    const int64_t buckets = std::min<int64_t>(kHistBuckets, ceil_div(n, (int64_t)1 << shift));
    int64_t k = 0;
    while (k < buckets) {
      int64_t k2 = k;
      unsigned long long sum = 0;
      while (k2 < buckets && sum + hist[k2] <= (unsigned long long)cap) sum += hist[k2++];
      if (k2 == k) return set_error(DOBFS_ERR_OOM, "a source bucket exceeds the build chunk");
      const int64_t lo = k << shift, hi = std::min<int64_t>(n, k2 << shift);
      uint64_t* sorted = nullptr;
      int64_t mc = 0;
      DOBFS_TRY(chunk_keys(G, nullptr, lo, hi, b, ka, kb, cap, s, &sorted, &mc));
      DevBuf offc, rawc;
      DOBFS_TRY(offc.alloc(sizeof(int64_t) * (size_t)(hi - lo + 1), s));
      DOBFS_TRY(rawc.alloc(sizeof(int64_t) * (size_t)(hi - lo + 1), s));
      int64_t kept = 0;
      DOBFS_TRY(extract<int64_t>(sorted, mc, b, hi - lo, offc.as<int64_t>(), nullptr, s, &kept));
      k_row_starts<<<grid_for(hi - lo + 1), kThreads, 0, s>>>(sorted, mc, b, hi - lo, rawc.as<int64_t>());
      k_chunk_degrees<<<grid_for(hi - lo), kThreads, 0, s>>>(offc.as<int64_t>(), rawc.as<int64_t>(), hi - lo, lo,
                                                            deg.as<int32_t>(), rawdeg.as<int32_t>());
      DOBFS_CUDA_TRY(cudaGetLastError());
      DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
      k = k2;
    }
  }
  // renumbering from the degrees
  if (flags & (DOBFS_GRAPH_REINDEX | DOBFS_GRAPH_REINDEX_EXACT)) {
    DevBuf vk, vt;
    DOBFS_TRY(vk.alloc(sizeof(uint64_t) * (size_t)n, s));
    DOBFS_TRY(vt.alloc(sizeof(uint64_t) * (size_t)n, s));
    const int cls_bits = std::max(b, 6) + 1;
    const int exact = (flags & DOBFS_GRAPH_REINDEX_EXACT) ? 1 : 0;
    k_vertex_keys_deg<<<grid_for(n), kThreads, 0, s>>>(deg.as<int32_t>(), n, b, cls_bits, exact, vk.as<uint64_t>());
    DOBFS_CUDA_TRY(cudaGetLastError());
    uint64_t* vsorted = nullptr;
    DOBFS_TRY(radix_sort_u64(vk.as<uint64_t>(), vt.as<uint64_t>(), n, b + cls_bits, s, &vsorted));
    DOBFS_TRY(g->new2orig.alloc(sizeof(int32_t) * (size_t)n, s));
    DOBFS_TRY(g->orig2new.alloc(sizeof(int32_t) * (size_t)n, s));
    k_maps<<<grid_for(n), kThreads, 0, s>>>(vsorted, n, b, g->new2orig.as<int32_t>(), g->orig2new.as<int32_t>());
    DOBFS_CUDA_TRY(cudaGetLastError());
    g->reindexed = true;
  }
  // row offsets (final order) and raw-count prefix for the chunks of pass 2
  DevBuf dnew, rnew, rawpre;
  DOBFS_TRY(dnew.alloc(sizeof(int64_t) * (size_t)n, s));
  DOBFS_TRY(rnew.alloc(sizeof(int64_t) * (size_t)n, s));
  k_gather_counts<<<grid_for(n), kThreads, 0, s>>>(g->reindexed ? g->new2orig.as<int32_t>() : nullptr,
                                                  deg.as<int32_t>(), rawdeg.as<int32_t>(), n, dnew.as<int64_t>(),
                                                  rnew.as<int64_t>());
  DOBFS_CUDA_TRY(cudaGetLastError());
  deg.reset();
  rawdeg.reset();
  DOBFS_TRY(rawpre.alloc(sizeof(int64_t) * (size_t)(n + 1), s));
  int64_t raw_total = 0, nnz = 0;
  DOBFS_TRY(exclusive_scan<int64_t>(rnew.as<int64_t>(), n, rawpre.as<int64_t>(), s, &raw_total));
  rnew.reset();
  // nnz first (the offset width depends on it), then the offsets
  {
    DevBuf tmp;
    DOBFS_TRY(tmp.alloc(sizeof(int64_t) * (size_t)(n + 1), s));
    DOBFS_TRY(exclusive_scan<int64_t>(dnew.as<int64_t>(), n, tmp.as<int64_t>(), s, &nnz));
    g->nnz = nnz;
    g->off64 = (flags & DOBFS_GRAPH_OFFSETS64) || nnz > (int64_t)INT32_MAX;
    if (g->off64) {
      g->off = std::move(tmp);
    } else {
      DOBFS_TRY(g->off.alloc(sizeof(int32_t) * (size_t)(n + 1), s));
      DOBFS_TRY(exclusive_scan<int32_t>(dnew.as<int64_t>(), n, g->off.as<int32_t>(), s, &nnz));
    }
  }
  dnew.reset();
  DOBFS_TRY(g->cols.alloc(sizeof(int32_t) * (size_t)(nnz + 4), s));
  DOBFS_CUDA_TRY(cudaMemsetAsync(g->cols.as<int32_t>() + nnz, 0, sizeof(int32_t) * 4, s));
  // pass 2: the columns, chunk by chunk of final row IDs
  if (g->off64)
    DOBFS_TRY(chunked_fill<int64_t>(g, G, rawpre.as<int64_t>(), ka, kb, cap, s));
  else
    DOBFS_TRY(chunked_fill<int32_t>(g, G, rawpre.as<int64_t>(), ka, kb, cap, s));
  rawpre.reset();
  ka.reset();
  kb.reset();
  return g->off64 ? finish_stats<int64_t>(g, s) : finish_stats<int32_t>(g, s);
}

}  // namespace

int build_from_keys(dobfs_graph* g, DevBuf& keys, int64_t m, uint32_t flags, cudaStream_t s) {
  const int b = g->bits;
  const int nbits = 2 * b;
  DevBuf tmp;
  DOBFS_TRY(tmp.alloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(m, 1), s));
  uint64_t* sorted = nullptr;
  DOBFS_TRY(radix_sort_u64(keys.as<uint64_t>(), tmp.as<uint64_t>(), m, nbits, s, &sorted));
  uint64_t* other = (sorted == keys.as<uint64_t>()) ? tmp.as<uint64_t>() : keys.as<uint64_t>();

  if ((flags & DOBFS_GRAPH_VALIDATE) && !(flags & DOBFS_GRAPH_SYMMETRIZE) && m > 0) {
    DevBuf err;
    DOBFS_TRY(err.alloc(sizeof(int), s));
    DOBFS_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    k_check_sym<<<grid_for(m), kThreads, 0, s>>>(sorted, m, b, err.as<int>());
    int h = 0;
    DOBFS_CUDA_TRY(cudaMemcpyAsync(&h, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) return set_error(DOBFS_ERR_BAD_GRAPH, "input graph is not symmetric (VALIDATE)");
  }

  const int64_t n = g->n;
  if (flags & (DOBFS_GRAPH_REINDEX | DOBFS_GRAPH_REINDEX_EXACT)) {
    // degrees in original IDs
    DevBuf off0;
    DOBFS_TRY(off0.alloc(sizeof(int64_t) * (size_t)(n + 1), s));
    int64_t nnz0 = 0;
    DOBFS_TRY(extract<int64_t>(sorted, m, b, n, off0.as<int64_t>(), nullptr, s, &nnz0));
    // degree-sorted order
    DevBuf vk, vt;
    DOBFS_TRY(vk.alloc(sizeof(uint64_t) * (size_t)n, s));
    DOBFS_TRY(vt.alloc(sizeof(uint64_t) * (size_t)n, s));
    // class < 64 + 2^b <= 2^(max(b, 6) + 1)
    const int cls_bits = std::max(b, 6) + 1;
    const int exact = (flags & DOBFS_GRAPH_REINDEX_EXACT) ? 1 : 0;
    k_vertex_keys<<<grid_for(n), kThreads, 0, s>>>(off0.as<int64_t>(), n, b, cls_bits, exact, vk.as<uint64_t>());
    DOBFS_CUDA_TRY(cudaGetLastError());
    uint64_t* vsorted = nullptr;
    DOBFS_TRY(radix_sort_u64(vk.as<uint64_t>(), vt.as<uint64_t>(), n, b + cls_bits, s, &vsorted));
    DOBFS_TRY(g->new2orig.alloc(sizeof(int32_t) * (size_t)n, s));
    DOBFS_TRY(g->orig2new.alloc(sizeof(int32_t) * (size_t)n, s));
    k_maps<<<grid_for(n), kThreads, 0, s>>>(vsorted, n, b, g->new2orig.as<int32_t>(), g->orig2new.as<int32_t>());
    k_relabel<<<grid_for(m), kThreads, 0, s>>>(sorted, m, b, g->orig2new.as<int32_t>(), other);
    DOBFS_CUDA_TRY(cudaGetLastError());
    vk.reset();
    vt.reset();
    off0.reset();
    uint64_t* a = other;
    uint64_t* bb = sorted;
    DOBFS_TRY(radix_sort_u64(a, bb, m, nbits, s, &sorted));
    g->reindexed = true;
  }

  // final CSR
  int64_t nnz = 0;
  {
    DevBuf base;
    const int P = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * 4, ceil_div(m, 4096)));
    DOBFS_TRY(kept_bases(sorted, m, P, base, s, &nnz));
  }
  g->nnz = nnz;
  g->off64 = (flags & DOBFS_GRAPH_OFFSETS64) || nnz > (int64_t)INT32_MAX;
  // the other key buffer is free now: release it before allocating the columns
  if (sorted == keys.as<uint64_t>()) tmp.reset(); else { keys.reset(); }
  DOBFS_TRY(g->cols.alloc(sizeof(int32_t) * (size_t)(nnz + 4), s));
  DOBFS_CUDA_TRY(cudaMemsetAsync(g->cols.as<int32_t>() + nnz, 0, sizeof(int32_t) * 4, s));
  DOBFS_TRY(g->off.alloc((g->off64 ? 8 : 4) * (size_t)(n + 1), s));
  int64_t nnz2 = 0;
  if (g->off64) {
    DOBFS_TRY(extract<int64_t>(sorted, m, b, n, g->off.as<int64_t>(), g->cols.as<int32_t>(), s, &nnz2));
    DOBFS_TRY(finish_stats<int64_t>(g, s));
  } else {
    DOBFS_TRY(extract<int32_t>(sorted, m, b, n, g->off.as<int32_t>(), g->cols.as<int32_t>(), s, &nnz2));
    DOBFS_TRY(finish_stats<int32_t>(g, s));
  }
  if (nnz2 != nnz) return set_error(DOBFS_ERR_CUDA, "internal: entry count changed between passes");
  return DOBFS_OK;
}

// ---------------------------------------------------------------- adopting a stored CSR
// A CSR that did not come out of this library's build (a graph file) is
// checked for every invariant the build establishes before any kernel relies
// on it: offsets non-decreasing from 0 to n_entries, columns in range, rows
// strictly increasing (sorted, no duplicates) and free of self-loops, and,
// for a renumbered graph, degree classes non-increasing along the internal
// IDs (so the isolated vertices come last and the vertices of degree >= 2^k
// form a prefix) with new2orig a permutation.

constexpr int kErrOffsets = 1, kErrColumn = 2, kErrRowOrder = 4, kErrClassOrder = 8, kErrPerm = 16,
              kErrAsym = 32;

// One warp per row.
template <class OffT>
__global__ void __launch_bounds__(kThreads) k_check_stored(const OffT* __restrict__ off,
                                                           const int32_t* __restrict__ cols, int64_t n, int64_t nnz,
                                                           int check_class, int* __restrict__ err) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const unsigned lane = lane_id();
  int bad = 0;
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int64_t s = (int64_t)off[v], e = (int64_t)off[v + 1];
    if (s < 0 || s > e || e > nnz) {
      bad |= kErrOffsets;
      continue;
    }
    if (check_class && lane == 0 && v + 1 < n) {
      const int64_t e2 = (int64_t)off[v + 2];
      if (e2 >= e && degree_class((uint64_t)(e - s), false) < degree_class((uint64_t)(e2 - e), false))
        bad |= kErrClassOrder;
    }
    for (int64_t p = s + lane; p < e; p += 32) {
      const int32_t c = cols[p];
      if (c < 0 || c >= n)
        bad |= kErrColumn;
      else if (c == v || (p > s && cols[p - 1] >= c))
        bad |= kErrRowOrder;
    }
  }
  if (bad) atomicOr(err, bad);
}

// o2n = inverse of n2o; o2n must hold -1 everywhere on entry. A value out of
// range or taken twice means n2o is not a permutation.
__global__ void k_invert_checked(const int32_t* __restrict__ n2o, int64_t n, int32_t* __restrict__ o2n,
                                 int* __restrict__ err) {
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = n2o[i];
    if (x < 0 || x >= n)
      bad |= kErrPerm;
    else if (atomicExch(o2n + x, (int32_t)i) != -1)
      bad |= kErrPerm;
  }
  if (bad) atomicOr(err, bad);
}

// Every stored u -> v has v -> u (binary search in v's sorted row); one warp
// per row u. Runs only on a CSR that passed k_check_stored.
template <class OffT>
__global__ void __launch_bounds__(kThreads) k_check_symmetric(const OffT* __restrict__ off,
                                                              const int32_t* __restrict__ cols, int64_t n,
                                                              int* __restrict__ err) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  int bad = 0;
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    const int64_t s = (int64_t)off[u], e = (int64_t)off[u + 1];
    for (int64_t p = s + lane_id(); p < e; p += 32) {
      const int32_t v = cols[p];
      int64_t a = (int64_t)off[v], z = (int64_t)off[v + 1];
      while (a < z) {
        const int64_t mid = a + ((z - a) >> 1);
        if (cols[mid] < (int32_t)u) a = mid + 1; else z = mid;
      }
      if (a == (int64_t)off[v + 1] || cols[a] != (int32_t)u) bad |= kErrAsym;
    }
  }
  if (bad) atomicOr(err, bad);
}

template <class OffT>
int adopt_checks(dobfs_graph* g, bool symmetric, cudaStream_t s, DevBuf& err, int* h) {
  const OffT* off = g->off.as<OffT>();
  const int32_t* cols = g->cols.as<int32_t>();
  const int grid = grid_for(g->n * 32);
  k_check_stored<OffT><<<grid, kThreads, 0, s>>>(off, cols, g->n, g->nnz, g->reindexed ? 1 : 0, err.as<int>());
  if (g->reindexed) {
    DOBFS_CUDA_TRY(cudaMemsetAsync(g->orig2new.ptr, 0xFF, sizeof(int32_t) * (size_t)g->n, s));
    k_invert_checked<<<grid_for(g->n), kThreads, 0, s>>>(g->new2orig.as<int32_t>(), g->n,
                                                         g->orig2new.as<int32_t>(), err.as<int>());
  }
  DOBFS_CUDA_TRY(cudaGetLastError());
  DOBFS_TRY(read_err_flag(err, s, h));
  if (*h == 0 && symmetric) {
    k_check_symmetric<OffT><<<grid, kThreads, 0, s>>>(off, cols, g->n, err.as<int>());
    DOBFS_CUDA_TRY(cudaGetLastError());
    DOBFS_TRY(read_err_flag(err, s, h));
  }
  return DOBFS_OK;
}

int adopt_csr(dobfs_graph* g, bool check_symmetric, cudaStream_t s) {
  const int64_t n = g->n;
  int64_t ends[2] = {0, 0};
  if (g->off64) {
    DOBFS_CUDA_TRY(cudaMemcpyAsync(&ends[0], g->off.as<int64_t>(), 8, cudaMemcpyDeviceToHost, s));
    DOBFS_CUDA_TRY(cudaMemcpyAsync(&ends[1], g->off.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, s));
    DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    int32_t e2[2] = {0, 0};
    DOBFS_CUDA_TRY(cudaMemcpyAsync(&e2[0], g->off.as<int32_t>(), 4, cudaMemcpyDeviceToHost, s));
    DOBFS_CUDA_TRY(cudaMemcpyAsync(&e2[1], g->off.as<int32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
    DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
    ends[0] = e2[0];
    ends[1] = e2[1];
  }
  if (ends[0] != 0 || ends[1] != g->nnz)
    return set_error(DOBFS_ERR_BAD_GRAPH, "stored row offsets must start at 0 and end at n_entries");
  DevBuf err;
  DOBFS_TRY(err.alloc(sizeof(int), s));
  DOBFS_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
  int h = 0;
  if (g->off64)
    DOBFS_TRY(adopt_checks<int64_t>(g, check_symmetric, s, err, &h));
  else
    DOBFS_TRY(adopt_checks<int32_t>(g, check_symmetric, s, err, &h));
  if (h & kErrOffsets) return set_error(DOBFS_ERR_BAD_GRAPH, "stored row offsets are not non-decreasing");
  if (h & kErrColumn) return set_error(DOBFS_ERR_BAD_GRAPH, "stored column out of range [0, %lld)", (long long)n);
  if (h & kErrRowOrder)
    return set_error(DOBFS_ERR_BAD_GRAPH, "a stored row is not strictly increasing or holds a self-loop");
  if (h & kErrClassOrder)
    return set_error(DOBFS_ERR_BAD_GRAPH, "renumbered graph: degree classes increase along the internal IDs");
  if (h & kErrPerm) return set_error(DOBFS_ERR_BAD_GRAPH, "renumbered graph: new2orig is not a permutation");
  if (h & kErrAsym) return set_error(DOBFS_ERR_BAD_GRAPH, "stored graph is not symmetric (VALIDATE)");
  return g->off64 ? finish_stats<int64_t>(g, s) : finish_stats<int32_t>(g, s);
}

int new_graph(int64_t n, cudaStream_t s, dobfs_graph** out) {
  if (!out) return set_error(DOBFS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > (int64_t)INT32_MAX)
    return set_error(DOBFS_ERR_INVALID, "n_vertices must be in [1, 2^31-1], got %lld", (long long)n);
  dobfs_graph* g = new (std::nothrow) dobfs_graph();
  if (!g) return set_error(DOBFS_ERR_OOM, "host allocation failed");
  g->n = n;
  g->bits = std::max(1, bits_for(n));
  g->stream = s;
  *out = g;
  return DOBFS_OK;
}

// Finishes a build: workspace, timing; on failure frees the graph.
int finish_graph(dobfs_graph* g, int rc, cudaEvent_t e0, cudaEvent_t e1, dobfs_graph** out) {
  if (rc == DOBFS_OK) rc = graph_alloc_workspace(g);
  if (rc == DOBFS_OK && e0 && e1) {
    cudaEventRecord(e1, g->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&g->build_ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc != DOBFS_OK) {
    graph_release(g);
    delete g;
    *out = nullptr;
    return rc;
  }
  *out = g;
  return DOBFS_OK;
}

int start_timer(cudaStream_t s, cudaEvent_t* e0, cudaEvent_t* e1) {
  *e0 = *e1 = nullptr;
  DOBFS_CUDA_TRY(cudaEventCreate(e0));
  DOBFS_CUDA_TRY(cudaEventCreate(e1));
  DOBFS_CUDA_TRY(cudaEventRecord(*e0, s));
  return DOBFS_OK;
}

int read_err_flag(DevBuf& err, cudaStream_t s, int* h) {
  DOBFS_CUDA_TRY(cudaMemcpyAsync(h, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  return DOBFS_OK;
}

namespace {

// Device copy of a caller array (host or device); `dev` stays empty when the
// caller's pointer is already device memory.
int to_device(const void* p, size_t bytes, bool device_ptrs, DevBuf& dev, cudaStream_t s, const void** out) {
  if (bytes == 0) {
    *out = p;
    return DOBFS_OK;
  }
  if (device_ptrs || is_device_ptr(p)) {
    *out = p;
    return DOBFS_OK;
  }
  DOBFS_TRY(dev.alloc(bytes, s));
  DOBFS_CUDA_TRY(cudaMemcpyAsync(dev.ptr, p, bytes, cudaMemcpyHostToDevice, s));
  *out = dev.ptr;
  return DOBFS_OK;
}

}  // namespace

}  // namespace dobfs

using namespace dobfs;

extern "C" {

int dobfs_graph_create_from_pairs(const int32_t* src, const int32_t* dst, int64_t n_pairs, int64_t n_vertices,
                                  uint32_t flags, void* stream, dobfs_graph** out) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (n_pairs < 0 || (n_pairs > 0 && (!src || !dst)))
    return set_error(DOBFS_ERR_INVALID, "bad pair arrays");
  dobfs_graph* g = nullptr;
  DOBFS_TRY(new_graph(n_vertices, s, &g));
  cudaEvent_t e0, e1;
  int rc = start_timer(s, &e0, &e1);
  if (rc == DOBFS_OK) {
    rc = [&]() -> int {
      DevBuf ds, dd, keys, err;
      const void *ps = nullptr, *pd = nullptr;
      const bool dp = (flags & DOBFS_GRAPH_DEVICE_PTRS) != 0;
      DOBFS_TRY(to_device(src, sizeof(int32_t) * (size_t)n_pairs, dp, ds, s, &ps));
      DOBFS_TRY(to_device(dst, sizeof(int32_t) * (size_t)n_pairs, dp, dd, s, &pd));
      const int64_t m = 2 * n_pairs;
      DOBFS_TRY(keys.alloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(m, 1), s));
      DOBFS_TRY(err.alloc(sizeof(int), s));
      DOBFS_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
      if (n_pairs > 0)
        k_keys_pairs<<<grid_for(n_pairs), kThreads, 0, s>>>((const int32_t*)ps, (const int32_t*)pd, n_pairs,
                                                            n_vertices, g->bits, keys.as<uint64_t>(), err.as<int>());
      DOBFS_CUDA_TRY(cudaGetLastError());
      int h = 0;
      DOBFS_TRY(read_err_flag(err, s, &h));
      if (h) return set_error(DOBFS_ERR_BAD_GRAPH, "pair endpoint out of range [0, %lld)", (long long)n_vertices);
      ds.reset();
      dd.reset();
      return build_from_keys(g, keys, m, flags | DOBFS_GRAPH_SYMMETRIZE, s);
    }();
  }
  return finish_graph(g, rc, e0, e1, out);
}

int dobfs_graph_create(const void* row_offsets, int offsets_are_int64, const int32_t* col_indices,
                       int64_t n_vertices, int64_t n_entries, uint32_t flags, void* stream, dobfs_graph** out) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (!row_offsets || n_entries < 0 || (n_entries > 0 && !col_indices))
    return set_error(DOBFS_ERR_INVALID, "bad CSR arrays");
  dobfs_graph* g = nullptr;
  DOBFS_TRY(new_graph(n_vertices, s, &g));
  cudaEvent_t e0, e1;
  int rc = start_timer(s, &e0, &e1);
  if (rc == DOBFS_OK) {
    rc = [&]() -> int {
      const bool dp = (flags & DOBFS_GRAPH_DEVICE_PTRS) != 0;
      const size_t ob = (offsets_are_int64 ? 8 : 4) * (size_t)(n_vertices + 1);
      DevBuf doff, dcol, keys, err;
      const void *po = nullptr, *pc = nullptr;
      DOBFS_TRY(to_device(row_offsets, ob, dp, doff, s, &po));
      DOBFS_TRY(to_device(col_indices, sizeof(int32_t) * (size_t)n_entries, dp, dcol, s, &pc));
      // first and last offsets must be 0 and n_entries
      int64_t ends[2] = {0, 0};
      if (offsets_are_int64) {
        DOBFS_CUDA_TRY(cudaMemcpyAsync(&ends[0], po, 8, cudaMemcpyDeviceToHost, s));
        DOBFS_CUDA_TRY(cudaMemcpyAsync(&ends[1], (const int64_t*)po + n_vertices, 8, cudaMemcpyDeviceToHost, s));
      } else {
        int32_t e2[2] = {0, 0};
        DOBFS_CUDA_TRY(cudaMemcpyAsync(&e2[0], po, 4, cudaMemcpyDeviceToHost, s));
        DOBFS_CUDA_TRY(cudaMemcpyAsync(&e2[1], (const int32_t*)po + n_vertices, 4, cudaMemcpyDeviceToHost, s));
        DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
        ends[0] = e2[0];
        ends[1] = e2[1];
      }
      DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
      if (ends[0] != 0 || ends[1] != n_entries)
        return set_error(DOBFS_ERR_BAD_GRAPH, "row offsets must start at 0 and end at n_entries");
      const int sym = (flags & DOBFS_GRAPH_SYMMETRIZE) ? 1 : 0;
      const int64_t m = n_entries * (sym ? 2 : 1);
      DOBFS_TRY(keys.alloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(m, 1), s));
      DOBFS_TRY(err.alloc(sizeof(int), s));
      DOBFS_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
      const int grid = grid_for(n_vertices * 32);
      if (offsets_are_int64)
        k_keys_csr<int64_t><<<grid, kThreads, 0, s>>>((const int64_t*)po, (const int32_t*)pc, n_vertices, n_entries,
                                                      g->bits, sym, keys.as<uint64_t>(), err.as<int>());
      else
        k_keys_csr<int32_t><<<grid, kThreads, 0, s>>>((const int32_t*)po, (const int32_t*)pc, n_vertices, n_entries,
                                                      g->bits, sym, keys.as<uint64_t>(), err.as<int>());
      DOBFS_CUDA_TRY(cudaGetLastError());
      int h = 0;
      DOBFS_TRY(read_err_flag(err, s, &h));
      if (h == 1) return set_error(DOBFS_ERR_BAD_GRAPH, "column index out of range [0, %lld)", (long long)n_vertices);
      if (h) return set_error(DOBFS_ERR_BAD_GRAPH, "row offsets are not non-decreasing within [0, n_entries]");
      doff.reset();
      dcol.reset();
      return build_from_keys(g, keys, m, flags, s);
    }();
  }
  return finish_graph(g, rc, e0, e1, out);
}

int dobfs_graph_create_rmat(int scale, int64_t n_pairs, uint32_t t_a, uint32_t t_ab, uint32_t t_abc, uint64_t seed,
                            uint32_t flags, void* stream, dobfs_graph** out) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (scale < 1 || scale > 31 || n_pairs < 0 || !(t_a <= t_ab && t_ab <= t_abc))
    return set_error(DOBFS_ERR_INVALID, "bad R-MAT parameters");
  dobfs_graph* g = nullptr;
  DOBFS_TRY(new_graph(int64_t(1) << scale, s, &g));
  cudaEvent_t e0, e1;
  int rc = start_timer(s, &e0, &e1);
  if (rc == DOBFS_OK) {
    rc = [&]() -> int {
      const int64_t m = 2 * n_pairs;
      // one-shot build: two 64-bit key buffers; chunked when they do not fit
      // next to the result (or when asked)
      size_t free_b = 0, total_b = 0;
      DOBFS_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
      const int64_t result_b = (int64_t)sizeof(int32_t) * m + 24 * (int64_t)g->n;
      const bool chunked = (flags & DOBFS_GRAPH_CHUNKED) || (16 * m + result_b > (int64_t)(0.9 * (double)free_b));
      if (chunked && n_pairs > 0) {
        RmatGen G{scale, n_pairs, t_a, t_ab, t_abc, gen_key_pairs(seed), gen_key_perm(seed)};
        int64_t cap = ((int64_t)(0.85 * (double)free_b) - result_b) / 16;
        if (cap < std::min<int64_t>(m, 1 << 16)) return set_error(DOBFS_ERR_OOM, "not enough device memory for a build chunk");
        if (flags & DOBFS_GRAPH_CHUNKED) cap = std::min<int64_t>(cap, std::max<int64_t>(1024, m / 7 + 1));  // several chunks
        cap = std::min<int64_t>(cap, m);
        return build_rmat_chunked(g, G, flags, cap, s);
      }
      DevBuf keys;
      DOBFS_TRY(keys.alloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(m, 1), s));
      if (n_pairs > 0)
        k_keys_rmat<<<grid_for(n_pairs), kThreads, 0, s>>>(n_pairs, scale, t_a, t_ab, t_abc, gen_key_pairs(seed),
                                                           gen_key_perm(seed), g->bits, keys.as<uint64_t>());
      DOBFS_CUDA_TRY(cudaGetLastError());
      return build_from_keys(g, keys, m, flags | DOBFS_GRAPH_SYMMETRIZE, s);
    }();
  }
  return finish_graph(g, rc, e0, e1, out);
}

int dobfs_graph_create_chunglu(const uint64_t* cdf, int64_t n_vertices, int64_t n_pairs, uint64_t seed,
                               uint32_t flags, void* stream, dobfs_graph** out) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (!cdf || n_pairs < 0) return set_error(DOBFS_ERR_INVALID, "bad Chung-Lu parameters");
  dobfs_graph* g = nullptr;
  DOBFS_TRY(new_graph(n_vertices, s, &g));
  cudaEvent_t e0, e1;
  int rc = start_timer(s, &e0, &e1);
  if (rc == DOBFS_OK) {
    rc = [&]() -> int {
      if (cdf[n_vertices - 1] == 0) return set_error(DOBFS_ERR_INVALID, "weight table sums to zero");
      DevBuf dcdf, keys;
      DOBFS_TRY(dcdf.alloc(sizeof(uint64_t) * (size_t)n_vertices, s));
      DOBFS_CUDA_TRY(cudaMemcpyAsync(dcdf.ptr, cdf, sizeof(uint64_t) * (size_t)n_vertices, cudaMemcpyHostToDevice, s));
      const int64_t m = 2 * n_pairs;
      DOBFS_TRY(keys.alloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(m, 1), s));
      if (n_pairs > 0)
        k_keys_chunglu<<<grid_for(n_pairs), kThreads, 0, s>>>(dcdf.as<uint64_t>(), (uint32_t)n_vertices, n_pairs,
                                                              gen_key_pairs(seed), gen_key_perm(seed), g->bits,
                                                              keys.as<uint64_t>());
      DOBFS_CUDA_TRY(cudaGetLastError());
      DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
      dcdf.reset();
      return build_from_keys(g, keys, m, flags | DOBFS_GRAPH_SYMMETRIZE, s);
    }();
  }
  return finish_graph(g, rc, e0, e1, out);
}

int dobfs_graph_export(const dobfs_graph* gc, int64_t* offsets_out, int32_t* cols_out, int32_t* new2orig_out,
                       void* stream) {
  clear_error();
  if (!gc) return set_error(DOBFS_ERR_INVALID, "graph is NULL");
  dobfs_graph* g = const_cast<dobfs_graph*>(gc);
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
  if (g->last_stream) DOBFS_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_done, 0));
  DevBuf tmp;
  if (offsets_out) {
    const size_t ob = sizeof(int64_t) * (size_t)(g->n + 1);
    int64_t* dst = offsets_out;
    const bool dev = is_device_ptr(offsets_out);
    if (!dev) {
      DOBFS_TRY(tmp.alloc(ob, s));
      dst = tmp.as<int64_t>();
    }
    if (g->off64)
      DOBFS_CUDA_TRY(cudaMemcpyAsync(dst, g->off.ptr, ob, cudaMemcpyDeviceToDevice, s));
    else
      k_widen<<<grid_for(g->n + 1), kThreads, 0, s>>>(g->off.as<int32_t>(), g->n + 1, dst);
    if (!dev) DOBFS_CUDA_TRY(cudaMemcpyAsync(offsets_out, dst, ob, cudaMemcpyDeviceToHost, s));
  }
  if (cols_out && g->nnz > 0)
    DOBFS_CUDA_TRY(cudaMemcpyAsync(cols_out, g->cols.ptr, sizeof(int32_t) * (size_t)g->nnz, cudaMemcpyDefault, s));
  if (new2orig_out) {
    if (g->reindexed) {
      DOBFS_CUDA_TRY(cudaMemcpyAsync(new2orig_out, g->new2orig.ptr, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDefault, s));
    } else {
      DevBuf id;
      int32_t* dst = new2orig_out;
      const bool dev = is_device_ptr(new2orig_out);
      if (!dev) {
        DOBFS_TRY(id.alloc(sizeof(int32_t) * (size_t)g->n, s));
        dst = id.as<int32_t>();
      }
      k_iota<<<grid_for(g->n), kThreads, 0, s>>>(dst, g->n);
      if (!dev) DOBFS_CUDA_TRY(cudaMemcpyAsync(new2orig_out, dst, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, s));
      DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
    }
  }
  DOBFS_CUDA_TRY(cudaGetLastError());
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  return DOBFS_OK;
}

int dobfs_graph_degrees(const dobfs_graph* gc, int32_t* deg_out, void* stream) {
  clear_error();
  if (!gc || !deg_out) return set_error(DOBFS_ERR_INVALID, "NULL argument");
  dobfs_graph* g = const_cast<dobfs_graph*>(gc);
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
  if (g->last_stream) DOBFS_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_done, 0));
  DevBuf tmp;
  int32_t* dst = deg_out;
  const bool dev = is_device_ptr(deg_out);
  if (!dev) {
    DOBFS_TRY(tmp.alloc(sizeof(int32_t) * (size_t)g->n, s));
    dst = tmp.as<int32_t>();
  }
  const int32_t* o2n = g->reindexed ? g->orig2new.as<int32_t>() : nullptr;
  if (g->off64)
    k_degrees<int64_t><<<grid_for(g->n), kThreads, 0, s>>>(g->off.as<int64_t>(), o2n, g->n, dst);
  else
    k_degrees<int32_t><<<grid_for(g->n), kThreads, 0, s>>>(g->off.as<int32_t>(), o2n, g->n, dst);
  DOBFS_CUDA_TRY(cudaGetLastError());
  if (!dev) DOBFS_CUDA_TRY(cudaMemcpyAsync(deg_out, dst, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, s));
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  return DOBFS_OK;
}

int dobfs_graph_wait(dobfs_graph* g, int32_t timeout_ms) {
  clear_error();
  if (!g) return set_error(DOBFS_ERR_INVALID, "graph is NULL");
  cudaEvent_t ev;
  {
    std::lock_guard<std::mutex> lk(g->mu);
    ev = g->ev_done;  // created with the run workspace, never replaced
  }
  if (!ev) return DOBFS_OK;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return DOBFS_OK;
    if (e != cudaErrorNotReady) return set_error(DOBFS_ERR_CUDA, "graph work failed: %s", cudaGetErrorString(e));
    if (timeout_ms >= 0 && std::chrono::steady_clock::now() - t0 >= std::chrono::milliseconds(timeout_ms))
      return set_error(DOBFS_ERR_TIMEOUT, "graph work still running after %d ms", timeout_ms);
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

int dobfs_graph_get_info(const dobfs_graph* g, dobfs_graph_info* info) {
  if (!g || !info) return set_error(DOBFS_ERR_INVALID, "NULL argument");
  info->n_vertices = g->n;
  info->n_entries = g->nnz;
  info->n_nonisolated = g->n_nonisolated;
  info->max_degree = g->max_degree;
  info->offsets_int64 = g->off64 ? 1 : 0;
  info->reindexed = g->reindexed ? 1 : 0;
  int64_t bytes = 0;
  const DevBuf* bufs[] = {&g->off, &g->cols, &g->new2orig, &g->orig2new, &g->isolated, &g->visited, &g->fbm,
                          &g->lp, &g->q0, &g->q1, &g->rec, &g->deferred, &g->firstdeg, &g->ctl, &g->trace,
                          &g->out_stage};
  for (const DevBuf* b : bufs) bytes += (int64_t)b->bytes;
  info->device_bytes = bytes;
  info->build_ms = g->build_ms;
  return DOBFS_OK;
}

}  // extern "C"
