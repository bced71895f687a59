// dobfs_run_static: a BFS entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a BFS:
// code that runs under a fixed memory budget that was reserved up front,
// allocation-free real-time or inference paths, or plugins hosted by a
// framework that owns all device allocations. dobfs_run needs a graph built
// by dobfs_graph_create, which allocates the CSR and a per-graph workspace.
// This entry point instead takes the caller's device CSR as it is and keeps
// all of its working memory (visited and frontier bitmaps, two frontier
// queues, a few counters) in one file-scope __device__ array of fixed size,
// so a call allocates nothing: no cudaMalloc, no cudaFree, no allocating
// library routine.
//
// The array lives on every GPU that loads this library, for the life of the
// process (kStaticBytes, about 8.4 MB). Host code never uses the array's
// name as a device address: every call, with the caller's device current,
// asks cudaGetSymbolAddress for the device address (a lookup, no
// allocation) and passes it to the kernels, so no address outlives the
// context it came from.
//
// The kernels are plain variants of the main path's: top-down expands one
// frontier vertex per thread, bottom-up scans one vertex's full row per
// thread (a warp owns one bitmap word), both with scalar loads, so the
// caller's column array needs no padding. Levels are chosen by the same
// alpha/beta rule on the host, one 32-byte counter read per level.
#include <cooperative_groups.h>

#include <mutex>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace dobfs {
namespace {

constexpr int64_t kStaticMaxVertices = DOBFS_STATIC_MAX_VERTICES;
constexpr int64_t kStaticWords = kStaticMaxVertices / 32;

struct StaticCtl {
  unsigned int q_tail;     // next-queue tail (top-down)
  unsigned int conv_tail;  // bitmap -> queue conversion tail
  unsigned long long nx_n; // vertices discovered by the step
  unsigned long long nx_m; // their degree sum
  int32_t bc_site;         // bounds-check builds: first failing check (0: none)
};

constexpr size_t kBitmapBytes = sizeof(uint32_t) * kStaticWords;
constexpr size_t kQueueBytes = sizeof(int32_t) * kStaticMaxVertices;
constexpr size_t kOffVisited = 0;
constexpr size_t kOffF0 = kOffVisited + kBitmapBytes;
constexpr size_t kOffF1 = kOffF0 + kBitmapBytes;
constexpr size_t kOffQ0 = kOffF1 + kBitmapBytes;
constexpr size_t kOffQ1 = kOffQ0 + kQueueBytes;
constexpr size_t kOffCtl = kOffQ1 + kQueueBytes;
constexpr size_t kStaticBytes = kOffCtl + 256;

// The working memory of dobfs_run_static, one copy per device.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct Scratch {
  uint32_t* visited;
  uint32_t* f[2];
  int32_t* q[2];
  StaticCtl* ctl;
};

constexpr int kThreads = 256;

__device__ __forceinline__ void st_enqueue(unsigned int* tail, int32_t* q, int32_t v, int64_t cap,
                                           int32_t* bc) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(tail, g.size());
  base = g.shfl(base, 0);
  if (bc_pos((int64_t)base + g.thread_rank(), cap, bc, kBcTdQueue)) q[base + g.thread_rank()] = v;
}

// Row bounds of u from the caller's offsets, clamped to [0, nnz] in
// bounds-check builds.
__device__ __forceinline__ void st_row(const int32_t* __restrict__ off, int32_t u, int64_t nnz, int32_t* bc,
                                       int site, int64_t& s, int64_t& e) {
  s = off[u];
  e = off[u + 1];
  bc_row(s, e, nnz, bc, site);
}

__global__ void k_st_clear(Scratch S, int64_t n, int64_t words, int32_t* __restrict__ level,
                           int32_t* __restrict__ parent) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n || i < words; i += stride) {
    if (i < words) {
      S.visited[i] = 0u;
      S.f[0][i] = 0u;
      S.f[1][i] = 0u;
    }
    if (i < n) {
      level[i] = -1;
      if (parent) parent[i] = -1;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S.ctl->q_tail = S.ctl->conv_tail = 0;
    S.ctl->nx_n = S.ctl->nx_m = 0;
    S.ctl->bc_site = 0;
  }
}

__global__ void k_st_seed(Scratch S, int32_t root, int32_t* __restrict__ level, int32_t* __restrict__ parent) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  S.visited[root >> 5] |= 1u << (root & 31);
  S.q[0][0] = root;
  level[root] = 0;
  if (parent) parent[root] = root;
}

// Top-down: one frontier vertex per thread; the first claim of a neighbour
// on the visited bitmap writes its level and parent and enqueues it.
__global__ void __launch_bounds__(kThreads) k_st_topdown(const int32_t* __restrict__ off,
                                                         const int32_t* __restrict__ cols, Scratch S, int32_t L,
                                                         int64_t nf, int64_t n, int64_t nnz,
                                                         int32_t* __restrict__ level,
                                                         int32_t* __restrict__ parent) {
  __shared__ unsigned long long sh[kThreads / 32];
  const int32_t* cur = S.q[L & 1];
  int32_t* nxt = S.q[(L + 1) & 1];
  int32_t* bc = &S.ctl->bc_site;
  unsigned long long m_new = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = bc_vid(cur[i], n, bc, kBcTdFrontier);
    int64_t s, e;
    st_row(off, u, nnz, bc, kBcTdRow, s, e);
    for (int64_t j = s; j < e; ++j) {
      const int32_t v = bc_vid(cols[j], n, bc, kBcTdColumn);
      const uint32_t bit = 1u << (v & 31);
      if (__ldcg(S.visited + (v >> 5)) & bit) continue;
      if (atomicOr(S.visited + (v >> 5), bit) & bit) continue;
      level[v] = L + 1;
      if (parent) parent[v] = u;
      int64_t vs, ve;
      st_row(off, v, nnz, bc, kBcTdRow, vs, ve);
      m_new += (unsigned long long)(ve - vs);
      st_enqueue(&S.ctl->q_tail, nxt, v, n, bc);
    }
  }
  m_new = block_sum_u64(m_new, sh);
  if (threadIdx.x == 0 && m_new) atomicAdd(&S.ctl->nx_m, m_new);
}

// Bottom-up: a warp owns one visited word; every unvisited vertex scans its
// row in order and stops at the first neighbour in the frontier.
__global__ void __launch_bounds__(kThreads) k_st_bottomup(const int32_t* __restrict__ off,
                                                          const int32_t* __restrict__ cols, Scratch S, int32_t L,
                                                          int64_t n, int64_t nnz, int64_t words,
                                                          int32_t* __restrict__ level,
                                                          int32_t* __restrict__ parent) {
  __shared__ unsigned long long sh[kThreads / 32];
  const uint32_t* front = S.f[L & 1];
  uint32_t* next = S.f[(L + 1) & 1];
  int32_t* bc = &S.ctl->bc_site;
  const unsigned lane = lane_id();
  unsigned long long n_new = 0, m_new = 0;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < words; w += warps) {
    const uint32_t vis = S.visited[w];
    const int64_t v = w * 32 + lane;
    bool found = false;
    int64_t d = 0;
    if (v < n && !((vis >> lane) & 1u)) {
      int64_t s, e;
      st_row(off, (int32_t)v, nnz, bc, kBcBuRow, s, e);
      d = e - s;
      for (int64_t j = s; j < e; ++j) {
        const int32_t u = bc_vid(cols[j], n, bc, kBcBuColumn);
        if ((front[u >> 5] >> (u & 31)) & 1u) {
          level[v] = L + 1;
          if (parent) parent[v] = u;
          found = true;
          break;
        }
      }
    }
    const unsigned fm = __ballot_sync(0xffffffffu, found);
    if (lane == 0) {
      next[w] = fm;
      if (fm) S.visited[w] = vis | fm;
      n_new += (unsigned)__popc(fm);
    }
    if (found) m_new += (unsigned long long)d;
  }
  n_new = block_sum_u64(n_new, sh);
  m_new = block_sum_u64(m_new, sh);
  if (threadIdx.x == 0) {
    if (n_new) atomicAdd(&S.ctl->nx_n, n_new);
    if (m_new) atomicAdd(&S.ctl->nx_m, m_new);
  }
}

__global__ void k_st_queue_to_bitmap(Scratch S, int32_t L, int64_t nf, int64_t n) {
  uint32_t* bm = S.f[L & 1];
  const int32_t* q = S.q[L & 1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = bc_vid(q[i], n, &S.ctl->bc_site, kBcConvert);
    atomicOr(bm + (v >> 5), 1u << (v & 31));
  }
}

__global__ void k_st_bitmap_to_queue(Scratch S, int32_t L, int64_t n, int64_t words) {
  const uint32_t* bm = S.f[L & 1];
  int32_t* q = S.q[L & 1];
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x = bm[w];
    if (!x) continue;
    unsigned pos = atomicAdd(&S.ctl->conv_tail, (unsigned)__popc(x));
    while (x) {
      const int b = __ffs(x) - 1;
      x &= x - 1;
      if (bc_pos(pos, n, &S.ctl->bc_site, kBcConvert)) q[pos] = (int32_t)(w * 32 + b);
      ++pos;
    }
  }
}

// Calls are serialised: they share the one array per device.
std::mutex g_static_mu;

// Device address of g_static_scratch on the current device. Looked up on
// every call (a lookup, not an allocation), so an address never outlives the
// context it belongs to (a cudaDeviceReset between calls is harmless).
int static_scratch(Scratch* S) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p)
    return set_error(DOBFS_ERR_CUDA, "cudaGetSymbolAddress(static scratch) failed: %s", cudaGetErrorString(e));
  unsigned char* b = static_cast<unsigned char*>(p);
  S->visited = reinterpret_cast<uint32_t*>(b + kOffVisited);
  S->f[0] = reinterpret_cast<uint32_t*>(b + kOffF0);
  S->f[1] = reinterpret_cast<uint32_t*>(b + kOffF1);
  S->q[0] = reinterpret_cast<int32_t*>(b + kOffQ0);
  S->q[1] = reinterpret_cast<int32_t*>(b + kOffQ1);
  S->ctl = reinterpret_cast<StaticCtl*>(b + kOffCtl);
  return DOBFS_OK;
}

}  // namespace
}  // namespace dobfs

using namespace dobfs;

extern "C" int dobfs_run_static(const int32_t* row_offsets, const int32_t* col_indices, int32_t n_vertices,
                                int32_t root, int32_t* level_out, int32_t* parent_out, void* stream) {
  clear_error();
  if (!row_offsets || !col_indices || !level_out)
    return set_error(DOBFS_ERR_INVALID, "dobfs_run_static: row_offsets, col_indices and level_out are required");
  if (n_vertices < 1 || (int64_t)n_vertices > kStaticMaxVertices)
    return set_error(DOBFS_ERR_INVALID,
                     "dobfs_run_static: n_vertices %d outside [1, %lld], the size of the static working memory",
                     n_vertices, (long long)kStaticMaxVertices);
  if (root < 0 || root >= n_vertices)
    return set_error(DOBFS_ERR_INVALID, "dobfs_run_static: root %d out of range [0, %d)", root, n_vertices);
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_static_mu);
  Scratch S;
  DOBFS_TRY(static_scratch(&S));

  const int64_t n = n_vertices;
  const int64_t words = ceil_div(n, 32);
  const int grid = sm_count() * 4;
  int32_t rowb[2] = {0, 0};
  int32_t nnz = 0;
  DOBFS_CUDA_TRY(cudaMemcpyAsync(rowb, row_offsets + root, sizeof(rowb), cudaMemcpyDeviceToHost, s));
  DOBFS_CUDA_TRY(cudaMemcpyAsync(&nnz, row_offsets + n, sizeof(nnz), cudaMemcpyDeviceToHost, s));
  k_st_clear<<<grid, kThreads, 0, s>>>(S, n, words, level_out, parent_out);
  k_st_seed<<<1, 32, 0, s>>>(S, root, level_out, parent_out);
  DOBFS_CUDA_TRY(cudaGetLastError());
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));

  // the alpha/beta rule with the library's defaults
  const int64_t alpha = 14, beta = 24;
  int64_t n_f = 1, m_f = rowb[1] - rowb[0], n_f_prev = 0, m_u = (int64_t)nnz - m_f;
  int dir = 0, fmt = 0;  // fmt: frontier held as 0 queue / 1 bitmap
  for (int32_t L = 0; n_f > 0; ++L) {
    if (L > 0) {
      if (dir == 0) dir = (m_f * alpha > m_u) ? 1 : 0;
      else dir = (n_f * beta < n && n_f < n_f_prev) ? 0 : 1;
    }
    if (dir == 0) {
      if (fmt == 1) k_st_bitmap_to_queue<<<grid, kThreads, 0, s>>>(S, L, n, words);
      k_st_topdown<<<grid, kThreads, 0, s>>>(row_offsets, col_indices, S, L, n_f, n, nnz, level_out, parent_out);
    } else {
      if (fmt == 0) {
        DOBFS_CUDA_TRY(cudaMemsetAsync(S.f[L & 1], 0, sizeof(uint32_t) * (size_t)words, s));
        k_st_queue_to_bitmap<<<grid, kThreads, 0, s>>>(S, L, n_f, n);
      }
      k_st_bottomup<<<grid, kThreads, 0, s>>>(row_offsets, col_indices, S, L, n, nnz, words, level_out,
                                              parent_out);
    }
    DOBFS_CUDA_TRY(cudaGetLastError());
    StaticCtl c;
    DOBFS_CUDA_TRY(cudaMemcpyAsync(&c, S.ctl, sizeof(c), cudaMemcpyDeviceToHost, s));
    DOBFS_CUDA_TRY(cudaMemsetAsync(S.ctl, 0, sizeof(StaticCtl), s));
    DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
    if (c.bc_site)
      return set_error(DOBFS_ERR_BOUNDS, "dobfs_run_static: device bounds check failed: %s",
                       bounds_site_name(c.bc_site));
    const int64_t n_new = (dir == 0) ? (int64_t)c.q_tail : (int64_t)c.nx_n;
    m_u -= (int64_t)c.nx_m;
    n_f_prev = n_f;
    n_f = n_new;
    m_f = (int64_t)c.nx_m;
    fmt = dir;
  }
  return DOBFS_OK;
}
