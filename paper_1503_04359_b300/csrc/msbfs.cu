// Bit-parallel multi-source BFS: up to 128 BFS (one per lane) over the same
// graph in one traversal, each vertex carrying lane masks of one or two
// 64-bit words (64 or 128 lanes per group), a vertex's words side by side.
//
//   seen[v]       lanes that have reached v
//   front/next    lanes for which v is in the current / next frontier
//   planes[b][v]  bit b of the iteration at which each lane reached v
//
// Where a step scans whole rows anyway (the wide bottom-up iterations, in
// which some live lane is nearly always still missing), its cost does not
// depend on the number of lanes, so a 128-lane group does the work of two
// 64-lane groups at about the cost of one.
//
// A step expands the frontier of iteration t for every lane at once, in the
// direction of Algorithm 1 picked by the same alpha/beta rule on the union of
// the lanes' frontiers:
//   top-down  every frontier vertex u pushes front[u] & ~seen[v] to each
//             neighbour v (atomicOr into next[v]);
//   bottom-up every vertex v still missing live lanes ORs front[u] over its
//             row and stops as soon as all the lanes it misses are found.
// Vertices found at iteration t+1 get seen |= new and the bits of t+1 set in
// the planes for those lanes, so each (lane, vertex) level costs no separate
// store; the flush writes level = (iteration found - start of lane) for all
// lanes of a vertex in one pass over original IDs, with coalesced stores per
// lane. Iterations are kept mod 2^16, so a lane may run at most 65535 levels.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../dobfs_inputs/gen.h"
#include "msbfs.cuh"

namespace cg = cooperative_groups;

namespace dobfs {
namespace {

constexpr int kThreads = 256;
constexpr int kMsChunk = 1024;  // top-down chunk record length (default; a run may set another)
constexpr int kMsT = 32;        // bottom-up entries per thread before a row continues warp-wide (default)
constexpr int kMsChunkMin = 256;
constexpr int kMsLongChunk = 4096;  // entries of a long bottom-up row per warp (chunk record)
constexpr int kMsCases = 3;
constexpr int kMsCaseNone = 7;
constexpr unsigned kIterMask = (1u << kMsPlanes) - 1u;
constexpr int kFirstPlanes = 4;  // planes cleared by a reset: iterations below 16

template <class OffT>
struct MsArgs {
  const OffT* off;
  const int32_t* cols;
  const int2* firstdeg;
  const int32_t* o2n;
  uint64_t* seen;   // [n][W]
  uint64_t* fb0;    // [n][W]
  uint64_t* fb1;    // [n][W]
  uint64_t* planes; // [kMsPlanes][n][W]
  int2* rec;
  int32_t* def;
  MsCtl* ctl;
  MsLaneStats* ls;
  const int64_t* small_tab;  // [2 * kSmallDeg]: row offset and first ID of each small degree (renumbered graphs)
  int32_t small_deg;         // degrees below this use small_tab for the row start (0: none)
  int64_t n, nnz, n_cand, rec_cap;
};

struct SeedArgs {
  int32_t count;
  int32_t lane[kMsLanes];
  int32_t root[kMsLanes];
};

// One mask word's flush: lanes of word `word` (bit i = lane 64 * word + i).
struct FlushArgs {
  unsigned long long lanes;
  int32_t word;
  int32_t release;
  int32_t vec;  // n % 4 == 0 and every flushed output row 16-byte aligned
  int32_t* out[kMsWordLanes];
  int32_t start[kMsWordLanes];
};

// The lane masks of one vertex: W words (64 lanes each), stored contiguously
// so that one access moves all of a vertex's lanes.
template <int W>
struct Lanes {
  unsigned long long w[W];
};

template <int W>
__device__ __forceinline__ Lanes<W> ld_lanes(const uint64_t* p, int64_t v) {
  Lanes<W> m;
  if constexpr (W == 2) {
    const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(p + 2 * v);
    m.w[0] = x.x;
    m.w[1] = x.y;
  } else {
    m.w[0] = p[v];
  }
  return m;
}

// through the read-only path (arrays not written during the kernel)
template <int W>
__device__ __forceinline__ Lanes<W> ldg_lanes(const uint64_t* p, int64_t v) {
  Lanes<W> m;
  if constexpr (W == 2) {
    const ulonglong2 x = __ldg(reinterpret_cast<const ulonglong2*>(p + 2 * v));
    m.w[0] = x.x;
    m.w[1] = x.y;
  } else {
    m.w[0] = __ldg(p + v);
  }
  return m;
}

// L2 only (words other threads update with atomics during the kernel)
template <int W>
__device__ __forceinline__ Lanes<W> ldcg_lanes(const uint64_t* p, int64_t v) {
  Lanes<W> m;
  if constexpr (W == 2) {
    const ulonglong2 x = __ldcg(reinterpret_cast<const ulonglong2*>(p + 2 * v));
    m.w[0] = x.x;
    m.w[1] = x.y;
  } else {
    m.w[0] = __ldcg(p + v);
  }
  return m;
}

template <int W>
__device__ __forceinline__ void st_lanes(uint64_t* p, int64_t v, const Lanes<W>& m) {
  if constexpr (W == 2) {
    *reinterpret_cast<ulonglong2*>(p + 2 * v) = make_ulonglong2(m.w[0], m.w[1]);
  } else {
    p[v] = m.w[0];
  }
}

template <int W>
__device__ __forceinline__ Lanes<W> zero_lanes() {
  Lanes<W> m;
#pragma unroll
  for (int i = 0; i < W; ++i) m.w[i] = 0ull;
  return m;
}

template <int W>
__device__ __forceinline__ bool any(const Lanes<W>& m) {
  unsigned long long x = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) x |= m.w[i];
  return x != 0ull;
}

template <int W>
__device__ __forceinline__ Lanes<W> and_not(const Lanes<W>& a, const Lanes<W>& b) {  // a & ~b
  Lanes<W> m;
#pragma unroll
  for (int i = 0; i < W; ++i) m.w[i] = a.w[i] & ~b.w[i];
  return m;
}

template <int W>
__device__ __forceinline__ Lanes<W> and_(const Lanes<W>& a, const Lanes<W>& b) {
  Lanes<W> m;
#pragma unroll
  for (int i = 0; i < W; ++i) m.w[i] = a.w[i] & b.w[i];
  return m;
}

template <int W>
__device__ __forceinline__ void or_into(Lanes<W>& a, const Lanes<W>& b) {
#pragma unroll
  for (int i = 0; i < W; ++i) a.w[i] |= b.w[i];
}

template <int W>
__device__ __forceinline__ bool covers(const Lanes<W>& acc, const Lanes<W>& need) {  // need is a subset of acc
  unsigned long long x = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) x |= need.w[i] & ~acc.w[i];
  return x == 0ull;
}

template <int W>
__device__ __forceinline__ Lanes<W> ctl_lanes(const unsigned long long* words) {
  Lanes<W> m;
#pragma unroll
  for (int i = 0; i < W; ++i) m.w[i] = words[i];
  return m;
}

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long x) {
  const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)x);
  const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(x >> 32));
  return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ void enqueue_ms(unsigned int* tail, int32_t* q, int32_t v, int64_t cap, int32_t* bc) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(tail, g.size());
  base = g.shfl(base, 0);
  if (bc_pos((int64_t)base + g.thread_rank(), cap, bc, kBcMsRecord)) q[base + g.thread_rank()] = v;
}

// Records the lanes `nw` found at vertex v at iteration T in the planes (one
// thread owns v).
template <int W, class OffT>
__device__ __forceinline__ void set_planes(const MsArgs<OffT>& A, int64_t v, const Lanes<W>& nw, unsigned T,
                                           int n_planes) {
  for (int b = 0; b < n_planes; ++b)
    if ((T >> b) & 1u) {
      Lanes<W> p = ld_lanes<W>(A.planes + (int64_t)b * A.n * W, v);
      or_into(p, nw);
      st_lanes<W>(A.planes + (int64_t)b * A.n * W, v, p);
    }
}

// Seeds lanes at their roots, one thread per seeded lane. A root is counted
// in the frontier and unvisited-edge totals once, by the first seed naming
// it, from the state before this seeding (read before any bit is set).
template <class OffT, int W>
__global__ void k_ms_seed(MsArgs<OffT> A, SeedArgs S) {
  const int i = threadIdx.x;
  MsCtl* c = A.ctl;
  const unsigned T = (unsigned)c->iter & kIterMask;
  const int np = c->n_planes;
  uint64_t* front = (c->iter & 1) ? A.fb1 : A.fb0;
  const bool mine = i < S.count;
  int32_t r = 0;
  bool s_old = false, f_old = false;
  if (mine) {
    r = A.o2n ? A.o2n[S.root[i]] : S.root[i];
    s_old = any(ld_lanes<W>(A.seen, r));
    f_old = any(ld_lanes<W>(front, r));
  }
  __syncthreads();
  if (mine) {
    const int l = S.lane[i], w = l / kMsWordLanes;
    const unsigned long long bit = 1ull << (l % kMsWordLanes);
    atomicOr(reinterpret_cast<unsigned long long*>(A.seen + (int64_t)r * W + w), bit);
    atomicOr(reinterpret_cast<unsigned long long*>(front + (int64_t)r * W + w), bit);
    for (int b = 0; b < np; ++b)
      if ((T >> b) & 1u)
        atomicOr(reinterpret_cast<unsigned long long*>(A.planes + (int64_t)b * A.n * W + (int64_t)r * W + w), bit);
    atomicOr(&c->active[w], bit);
    atomicOr(&c->live[w], bit);
    // a lane starts top-down, also when it joins after the switch chose this
    // step's directions (the server then runs both kinds of step)
    atomicAnd(&c->lane_bu[w], ~bit);
    atomicOr(&c->td_mask[w], bit);
    atomicAnd(&c->bu_mask[w], ~bit);
    bool first = true;
    for (int j = 0; j < i && first; ++j) first = S.root[j] != S.root[i];
    if (first) {
      const long long d = (long long)A.off[r + 1] - (long long)A.off[r];
      if (!f_old) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&c->n_f), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(&c->m_f), (unsigned long long)d);
      }
      if (!s_old) atomicAdd(reinterpret_cast<unsigned long long*>(&c->m_u), (unsigned long long)(-d));
    }
  }
}

__global__ void k_ms_set_ctl(MsCtl* dst, MsCtl c) { *dst = c; }

template <class OffT, int W>
__global__ void k_ms_switch(MsArgs<OffT> A, cudaGraphConditionalHandle h_while, cudaGraphConditionalHandle h_case,
                            int in_graph) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  MsCtl* c = A.ctl;
  if (!c->fresh) {
    // active vertices: the frontier vertices pushed top-down and the vertices searched bottom-up
    const int64_t act = (int64_t)c->nx_tdact + (int64_t)c->nx_act;
    c->alg_bytes += 16 * W * act + (8 * W + 4) * (int64_t)c->nx_examined;
    c->nx_act = c->nx_tdact = 0;
    c->n_f_prev = c->n_f;
    c->n_f = (int64_t)c->nx_n;
    c->m_f = (int64_t)c->nx_m;
    c->m_u -= (int64_t)c->nx_mu;
    for (int w = 0; w < W; ++w) {
      c->live[w] = c->nx_live[w] & c->active[w];
      c->nx_live[w] = 0;
    }
    c->examined += (int64_t)c->nx_examined;
    c->iter += 1;
    c->levels_run += 1;
    c->nx_n = c->nx_m = c->nx_mu = c->nx_examined = 0;
    c->n_rec = c->n_def = 0;
  }
  const int prev_dir = c->fresh ? 0 : c->dir;
  c->fresh = 0;
  // done: no lane can discover anything; the server may still seed new lanes
  // and run the step, so the direction is picked in any case
  // a graph-driven batch has fewer than n iterations: more can only come
  // from a fault in the step kernels, and ends the loop instead of running on
  const bool runaway = in_graph && (int64_t)c->levels_run > A.n;
  if (runaway) c->runaway = 1;
  unsigned long long any_live = 0;
  for (int w = 0; w < W; ++w) any_live |= c->live[w];
  const bool done = (any_live == 0 || c->n_f == 0 || runaway);
  if (done)
    for (int w = 0; w < W; ++w) c->live[w] = 0;
  // direction by lane: a top-down lane turns bottom-up by the alpha rule on
  // its own (sampled) frontier statistics, so that lanes whose frontier is
  // still small push it top-down while the others search bottom-up in the
  // same step (a bottom-up search for a lane with a small frontier scans
  // whole rows); bottom-up lanes return to top-down together, by the beta
  // rule on the union of the frontiers (late levels stay one kind of step)
  (void)prev_dir;
  unsigned long long was_any_bu = 0;
  for (int w = 0; w < W; ++w) was_any_bu |= c->lane_bu[w] & c->live[w];
  const bool union_to_td = was_any_bu && c->n_f * (int64_t)c->beta < A.n && c->n_f < c->n_f_prev;
  unsigned long long bu[kMsMaxWords] = {};
  for (int w = 0; w < W; ++w) {
    const unsigned long long lv = c->live[w];
    switch (c->mode) {
      case DOBFS_DIR_TOPDOWN: bu[w] = 0; break;
      case DOBFS_DIR_BOTTOMUP: bu[w] = lv; break;
      case DOBFS_DIR_RANDOM:  // a seeded coin per lane and step
        bu[w] = lv & gen_mix64(c->sched_seed ^ ((uint64_t)c->iter << 1) ^ ((uint64_t)w << 40));
        break;
      default:
        for (unsigned long long x = lv; x; x &= x - 1) {
          const int b = __ffsll((long long)x) - 1, l = w * kMsWordLanes + b;
          const int64_t mf = (int64_t)A.ls->m_f[l] * kMsLaneSample;
          const int64_t mu = (int64_t)A.ls->m_u[l] * kMsLaneSample;
          const bool was_bu = (c->lane_bu[w] >> b) & 1ull;
          const bool to_bu = was_bu ? !union_to_td : (mf * (int64_t)c->alpha > mu);
          if (to_bu) bu[w] |= 1ull << b;
        }
        break;
    }
  }
  bool any_td = false, any_bu = false;
  for (int l = 0; l < kMsLanes; ++l) {  // statistics of this step become the previous ones
    A.ls->n_f_prev[l] = A.ls->n_f[l];
    A.ls->n_f[l] = A.ls->m_f[l] = A.ls->m_u[l] = 0;
  }
  for (int w = 0; w < W; ++w) {
    c->bu_mask[w] = bu[w];
    c->td_mask[w] = c->live[w] & ~bu[w];
    c->lane_bu[w] = (c->lane_bu[w] & ~c->live[w]) | bu[w];
    any_td |= c->td_mask[w] != 0;
    any_bu |= bu[w] != 0;
  }
  const int dir = (any_td && any_bu) ? 2 : (any_bu ? 1 : 0);
  // the planes needed by iteration t+1 must be clean: clear the next one the
  // first time t+1 reaches it
  const unsigned tn = (unsigned)(c->iter + 1) & kIterMask;
  c->clear_plane = -1;
  if (c->n_planes < kMsPlanes && (tn >> c->n_planes) != 0u) {
    c->clear_plane = c->n_planes;
    c->n_planes += 1;
  }
  c->dir = dir;
  c->step_case = dir;
  c->done = done ? 1 : 0;
  if (in_graph) {
    if (done) {
      cudaGraphSetConditional(h_case, kMsCaseNone);
      cudaGraphSetConditional(h_while, 0);
    } else {
      cudaGraphSetConditional(h_case, (unsigned)dir);
    }
  }
}

// Per-lane frontier statistics for the direction switch (auto policy only),
// sampled from every kMsLaneSample-th block of 32 candidate vertices: for each
// lane, the sampled vertices in its frontier, their degree sum, and the
// degree sum of the sampled vertices it has not reached. Runs just before the
// switch, so the frontier is what the step before wrote (or the seeds). Skips
// the work while every lane is top-down and the rule on the union of the
// lanes says top-down: no single lane's rule can then say bottom-up (a lane's
// frontier is part of the union's, and its unreached part holds the union's).
template <class OffT, int W>
__global__ void __launch_bounds__(kThreads) k_ms_lane_stats(MsArgs<OffT> A) {
  const MsCtl* c = A.ctl;
  if (c->mode != DOBFS_DIR_AUTO) return;
  const int64_t m_f = c->fresh ? c->m_f : (int64_t)c->nx_m;
  const int64_t m_u = c->fresh ? c->m_u : c->m_u - (int64_t)c->nx_mu;
  unsigned long long any_bu = 0;
  for (int w = 0; w < W; ++w) any_bu |= c->lane_bu[w] & c->live[w];
  if (!any_bu && m_f * (int64_t)c->alpha <= m_u) return;
  __shared__ unsigned long long s_n[kMsWordLanes * W], s_m[kMsWordLanes * W], s_u[kMsWordLanes * W];
  for (int i = threadIdx.x; i < kMsWordLanes * W; i += blockDim.x) s_n[i] = s_m[i] = s_u[i] = 0;
  __syncthreads();
  // the frontier of the step about to be chosen (the switch that follows
  // advances the iteration unless no step ran since the seeds)
  const bool at_seed = c->fresh != 0;
  const uint64_t* front = (((c->iter & 1) != 0) == at_seed) ? A.fb1 : A.fb0;
  const unsigned lane = lane_id();
  const int64_t rounds = ceil_div(A.n_cand, 32);
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t r = gw * kMsLaneSample; r < rounds; r += warps * kMsLaneSample) {
    const int64_t v = r * 32 + lane;
    const bool in = v < A.n_cand;
    const Lanes<W> f = in ? ldg_lanes<W>(front, v) : zero_lanes<W>();
    const Lanes<W> sn = in ? ldg_lanes<W>(A.seen, v) : zero_lanes<W>();
    const unsigned d = in ? (unsigned)min(__ldg(&A.firstdeg[v].y), 1 << 26) : 0u;  // 32 of them fit 32 bits
#pragma unroll
    for (int w = 0; w < W; ++w)
#pragma unroll 4
      for (int b = 0; b < kMsWordLanes; ++b) {
        const bool fb = (f.w[w] >> b) & 1ull;
        const bool ub = in && !((sn.w[w] >> b) & 1ull);
        const unsigned cf = __ballot_sync(0xffffffffu, fb);
        const unsigned mf = __reduce_add_sync(0xffffffffu, fb ? d : 0u);
        const unsigned mu = __reduce_add_sync(0xffffffffu, ub ? d : 0u);
        if (lane == 0) {
          const int l = w * kMsWordLanes + b;
          if (cf) {
            atomicAdd(&s_n[l], (unsigned long long)__popc(cf));
            atomicAdd(&s_m[l], (unsigned long long)mf);
          }
          if (mu) atomicAdd(&s_u[l], (unsigned long long)mu);
        }
      }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kMsWordLanes * W; i += blockDim.x) {
    if (s_n[i]) atomicAdd(&A.ls->n_f[i], s_n[i]);
    if (s_m[i]) atomicAdd(&A.ls->m_f[i], s_m[i]);
    if (s_u[i]) atomicAdd(&A.ls->m_u[i], s_u[i]);
  }
}

// Between the top-down and bottom-up halves of a step with lanes of both
// directions: the chunk records of the top-down push are done with, and the
// bottom-up search counts its own from zero.
template <class OffT, int W>
__global__ void k_ms_reset_records(MsArgs<OffT> A) {
  if (threadIdx.x == 0 && blockIdx.x == 0) A.ctl->n_rec = 0;
}

// Restarts the iteration count of a group none of whose lanes holds a query.
// The releasing flushes cleared every lane's bits in the planes in use, so
// all planes are clean; planes from kFirstPlanes up are cleared again when an
// iteration first needs them. Discovery iterations then stay small: fewer
// plane bits to set per discovery and fewer planes per flush.
template <class OffT, int W>
__global__ void k_ms_rebase(MsArgs<OffT> A) {
  MsCtl* c = A.ctl;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int w = 0; w < W; ++w)
    if (c->active[w] != 0) return;
  c->iter = 0;
  if (c->n_planes > kFirstPlanes) c->n_planes = kFirstPlanes;
  c->clear_plane = -1;
}

template <class OffT, int W>
__global__ void k_ms_clear_plane(MsArgs<OffT> A) {
  const int b = A.ctl->clear_plane;
  if (b < 0) return;
  uint64_t* p = A.planes + (int64_t)b * A.n * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n * W; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0ull;
}

template <class OffT, int W>
__global__ void k_ms_clear_next(MsArgs<OffT> A) {
  uint64_t* next = (A.ctl->iter & 1) ? A.fb0 : A.fb1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n_cand * W;
       i += (int64_t)gridDim.x * blockDim.x)
    next[i] = 0ull;
}

// Top-down, part 1: chunk records for the rows of the frontier vertices.
template <class OffT, int W>
__global__ void __launch_bounds__(kThreads) k_ms_td_list(MsArgs<OffT> A) {
  __shared__ unsigned long long sh[kThreads / 32];
  const uint64_t* front = (A.ctl->iter & 1) ? A.fb1 : A.fb0;
  const int64_t chunk = A.ctl->td_chunk;
  const Lanes<W> tdm = ctl_lanes<W>(A.ctl->td_mask);  // lanes expanded top-down
  unsigned long long act = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < A.n_cand; v += (int64_t)gridDim.x * blockDim.x) {
    if (!any(and_(ld_lanes<W>(front, v), tdm))) continue;
    act += 1;
    const int64_t d = (int64_t)A.off[v + 1] - (int64_t)A.off[v];
    if (d == 0) continue;
    const unsigned nch = (unsigned)ceil_div(d, chunk);
    const unsigned base = atomicAdd(&A.ctl->n_rec, nch);
    if ((int64_t)base + nch > A.rec_cap) continue;  // cannot happen: one record per kMsChunkMin entries or vertex
    for (unsigned k = 0; k < nch; ++k) A.rec[base + k] = make_int2((int32_t)v, (int32_t)k);
  }
  act = block_sum_u64(act, sh);
  if (threadIdx.x == 0 && act) atomicAdd(&A.ctl->nx_tdact, act);
}

// Top-down, part 2: one warp per record pushes front[u] to the unseen lanes
// of each neighbour.
template <class OffT, int W, int NT>
__global__ void __launch_bounds__(NT) k_ms_td(MsArgs<OffT> A) {
  __shared__ unsigned long long sh[NT / 32];
  const MsCtl* c = A.ctl;
  const uint64_t* front = (c->iter & 1) ? A.fb1 : A.fb0;
  uint64_t* next = (c->iter & 1) ? A.fb0 : A.fb1;
  const int64_t nrec = min((int64_t)c->n_rec, A.rec_cap);
  const int64_t chunk = c->td_chunk;
  const unsigned lane = lane_id();
  unsigned long long ex = 0;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < nrec; r += warps) {
    const int2 rc = A.rec[r];
    const int32_t u = bc_vid(rc.x, A.n, &A.ctl->bc_site, kBcMsRecord);
    const Lanes<W> fu = and_(ld_lanes<W>(front, u), ctl_lanes<W>(c->td_mask));
    int64_t ro = (int64_t)A.off[u], re = (int64_t)A.off[u + 1];
    bc_row(ro, re, A.nnz, &A.ctl->bc_site, kBcMsRow);
    const int64_t s = ro + (int64_t)rc.y * chunk;
    const int64_t e = min(re, s + chunk);
    if (lane == 0 && e > s) ex += (unsigned long long)(e - s);
    for (int64_t j = s + lane; j < e; j += 32) {
      const int32_t v = bc_vid(A.cols[j], A.n, &A.ctl->bc_site, kBcMsColumn);
      const Lanes<W> m = and_not(fu, ldg_lanes<W>(A.seen, v));
      if (!any(m)) continue;
      const Lanes<W> nx = ldcg_lanes<W>(next, v);
#pragma unroll
      for (int w = 0; w < W; ++w)
        if (m.w[w] & ~nx.w[w]) atomicOr(reinterpret_cast<unsigned long long*>(next + v * W + w), m.w[w]);
    }
  }
  ex = block_sum_u64(ex, sh);
  if (threadIdx.x == 0 && ex) atomicAdd(&A.ctl->nx_examined, ex);
}

// Folds the lanes found at vertex v into the step's counters.
template <int W>
struct MsCount {
  unsigned long long n = 0, m = 0, mu = 0, ex = 0, act = 0;
  unsigned long long live[W] = {};
};

template <int W>
__device__ __forceinline__ void ms_count_flush(MsCtl* c, MsCount<W>& k, unsigned long long* sh, bool with_ex) {
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const unsigned long long lv = warp_or64(k.live[w]);
    if (lane_id() == 0 && lv) atomicOr(&c->nx_live[w], lv);
  }
  k.n = block_sum_u64(k.n, sh);
  k.m = block_sum_u64(k.m, sh);
  k.mu = block_sum_u64(k.mu, sh);
  if (with_ex) {
    k.ex = block_sum_u64(k.ex, sh);
    k.act = block_sum_u64(k.act, sh);
  }
  if (threadIdx.x == 0) {
    if (k.n) atomicAdd(&c->nx_n, k.n);
    if (k.m) atomicAdd(&c->nx_m, k.m);
    if (k.mu) atomicAdd(&c->nx_mu, k.mu);
    if (with_ex && k.ex) atomicAdd(&c->nx_examined, k.ex);
    if (with_ex && k.act) atomicAdd(&c->nx_act, k.act);
  }
}

// Records lanes nw (non-empty) newly found at v: seen, planes, counters.
template <int W, class OffT>
__device__ __forceinline__ void ms_found(const MsArgs<OffT>& A, int64_t v, const Lanes<W>& s, const Lanes<W>& nw,
                                         int64_t deg, unsigned T, int np, MsCount<W>& k) {
  Lanes<W> s2 = s;
  or_into(s2, nw);
  st_lanes<W>(A.seen, v, s2);
  set_planes<W>(A, v, nw, T, np);
  k.n += 1;
  k.m += (unsigned long long)deg;
  if (!any(s)) k.mu += (unsigned long long)deg;
#pragma unroll
  for (int w = 0; w < W; ++w) k.live[w] |= nw.w[w];
}

// Top-down, part 3: the pushed masks become the next frontier; record them.
template <class OffT, int W>
__global__ void __launch_bounds__(kThreads) k_ms_td_post(MsArgs<OffT> A) {
  __shared__ unsigned long long sh[kThreads / 32];
  MsCtl* c = A.ctl;
  uint64_t* next = (c->iter & 1) ? A.fb0 : A.fb1;
  const unsigned T = (unsigned)(c->iter + 1) & kIterMask;
  const int np = c->n_planes;
  MsCount<W> k;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < A.n_cand; v += (int64_t)gridDim.x * blockDim.x) {
    const Lanes<W> nx = ld_lanes<W>(next, v);
    if (!any(nx)) continue;
    const Lanes<W> s = ld_lanes<W>(A.seen, v);
    const Lanes<W> nw = and_not(nx, s);
    st_lanes<W>(next, v, nw);
    if (!any(nw)) continue;
    ms_found<W>(A, v, s, nw, A.firstdeg[v].y, T, np, k);
  }
  ms_count_flush<W>(c, k, sh, false);
}

// Bottom-up, part 1: one vertex per thread. A vertex missing live lanes ORs
// the frontier masks of its first bu_scan neighbours and stops once every
// missing lane is found; longer rows continue in k_ms_bu_long with the
// partial mask kept in next[v].
// (at most 64 registers: 32 resident warps per SM at any block size)
template <class OffT, int W, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_ms_bu(MsArgs<OffT> A, int merge) {
  __shared__ unsigned long long sh[NT / 32];
  __shared__ int64_t s_tab[2 * kSmallDeg];
  if (threadIdx.x < 2 * kSmallDeg) s_tab[threadIdx.x] = A.small_deg ? A.small_tab[threadIdx.x] : 0;
  __syncthreads();
  MsCtl* c = A.ctl;
  const uint64_t* front = (c->iter & 1) ? A.fb1 : A.fb0;
  uint64_t* next = (c->iter & 1) ? A.fb0 : A.fb1;
  const Lanes<W> bum = ctl_lanes<W>(c->bu_mask);  // lanes searched bottom-up
  // merge (a step with lanes of both directions): next already holds the
  // top-down lanes' pushes, which this pass records with its own finds
  const unsigned T = (unsigned)(c->iter + 1) & kIterMask;
  const int np = c->n_planes;
  const int64_t scan = c->bu_scan;
  MsCount<W> k;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < A.n_cand; v += (int64_t)gridDim.x * blockDim.x) {
    const Lanes<W> s = ld_lanes<W>(A.seen, v);
    const Lanes<W> need = and_not(bum, s);
    const Lanes<W> pushed = merge ? and_not(ld_lanes<W>(next, v), s) : zero_lanes<W>();
    if (!any(need)) {
      st_lanes<W>(next, v, pushed);
      if (any(pushed)) ms_found<W>(A, v, s, pushed, A.firstdeg[v].y, T, np, k);
      continue;
    }
    k.act += 1;
    const int2 fd = A.firstdeg[v];
    Lanes<W> acc = zero_lanes<W>();
    int64_t j = 0;
    if (fd.y > 0) {
      acc = ldg_lanes<W>(front, bc_vid(fd.x, A.n, &A.ctl->bc_site, kBcMsColumn));
      j = 1;
      // small degrees: the row start follows from the ID (no offset load)
      int64_t o = fd.y < A.small_deg ? s_tab[fd.y] + (v - s_tab[kSmallDeg + fd.y]) * fd.y : (int64_t)A.off[v];
      int64_t oe = o + fd.y;
      bc_row(o, oe, A.nnz, &A.ctl->bc_site, kBcMsRow);
      const int64_t lim = min(oe - o, scan);
      while (j < lim && !covers(acc, need)) {
        int32_t u[4];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          u[t] = (j + t < lim) ? bc_vid(A.cols[o + j + t], A.n, &A.ctl->bc_site, kBcMsColumn) : -1;
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (u[t] >= 0) or_into(acc, ldg_lanes<W>(front, u[t]));
        j = min(j + 4, lim);
      }
    }
    k.ex += (unsigned long long)j;
    Lanes<W> nw = and_(acc, need);
    if (!covers(nw, need) && fd.y > scan) {
      // partial: k_ms_bu_long scans the rest of the row in chunk records,
      // k_ms_bu_fin then records the vertex
      or_into(nw, pushed);
      st_lanes<W>(next, v, nw);
      enqueue_ms(&c->n_def, A.def, (int32_t)v, A.n, &c->bc_site);
      if ((int64_t)fd.y - scan > kMsLongChunk) {  // chunks after the first go to chunk records
        const unsigned nch = (unsigned)ceil_div((int64_t)fd.y - scan, (int64_t)kMsLongChunk);
        const unsigned base = atomicAdd(&c->n_rec, nch - 1);
        for (unsigned r = 1; r < nch; ++r)
          if ((int64_t)base + r - 1 < A.rec_cap) A.rec[base + r - 1] = make_int2((int32_t)v, (int32_t)r);
      }
      continue;
    }
    or_into(nw, pushed);
    st_lanes<W>(next, v, nw);
    if (!any(nw)) continue;
    ms_found<W>(A, v, s, nw, fd.y, T, np, k);
  }
  ms_count_flush<W>(c, k, sh, true);
}

// Bottom-up, part 2: the rest of the deferred rows, one warp per row for its
// first kMsLongChunk entries, then one warp per chunk record for the further
// chunks of longer rows (a hub row is spread over many warps). The records
// come after the rows in the work order, so a record usually starts once its
// row's first chunk is done: it skips if the lanes found so far (next[v],
// OR-ed in by every warp of the row) already cover the row, and re-checks
// every 1024 entries. Early-exit test after every 128 entries.
template <class OffT, int W>
__global__ void __launch_bounds__(kThreads) k_ms_bu_long(MsArgs<OffT> A) {
  __shared__ unsigned long long sh[kThreads / 32];
  MsCtl* c = A.ctl;
  const uint64_t* front = (c->iter & 1) ? A.fb1 : A.fb0;
  uint64_t* next = (c->iter & 1) ? A.fb0 : A.fb1;
  const Lanes<W> bum = ctl_lanes<W>(c->bu_mask);  // lanes searched bottom-up
  const int64_t nrec = min((int64_t)c->n_rec, A.rec_cap);
  const int64_t nd = c->n_def;
  const int64_t scan = c->bu_scan;
  const unsigned lane = lane_id();
  unsigned long long ex = 0;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < nd + nrec; i += warps) {
    int32_t v;
    int64_t s0, e0;
    if (i < nd) {  // a deferred row: the first chunk of the rest
      v = bc_vid(A.def[i], A.n, &c->bc_site, kBcMsRecord);
      int64_t o = (int64_t)A.off[v], e = (int64_t)A.off[v + 1];
      bc_row(o, e, A.nnz, &c->bc_site, kBcMsRow);
      s0 = o + scan;
      e0 = min(e, s0 + kMsLongChunk);
    } else {
      const int2 rc = A.rec[i - nd];
      v = bc_vid(rc.x, A.n, &c->bc_site, kBcMsRecord);
      int64_t o = (int64_t)A.off[v], e = (int64_t)A.off[v + 1];
      bc_row(o, e, A.nnz, &c->bc_site, kBcMsRow);
      s0 = o + scan + (int64_t)rc.y * kMsLongChunk;
      e0 = min(e, s0 + kMsLongChunk);
    }
    const Lanes<W> need = and_not(bum, ld_lanes<W>(A.seen, v));
    Lanes<W> acc = ldcg_lanes<W>(next, v);
    int step = 0;
    for (int64_t base = s0 & ~3ll; base < e0 && !covers(acc, need); base += 128, ++step) {
      if (i >= nd && (step & 7) == 7) {
        or_into(acc, ldcg_lanes<W>(next, v));  // what the row's other warps found
        if (covers(acc, need)) break;
      }
      const int64_t p = base + 4 * (int64_t)lane;
      Lanes<W> x = zero_lanes<W>();
      if (p < e0) {
        const int4 c4 = *reinterpret_cast<const int4*>(A.cols + p);
        const int32_t us[4] = {bc_vid(c4.x, A.n, &c->bc_site, kBcMsColumn), bc_vid(c4.y, A.n, &c->bc_site, kBcMsColumn),
                               bc_vid(c4.z, A.n, &c->bc_site, kBcMsColumn), bc_vid(c4.w, A.n, &c->bc_site, kBcMsColumn)};
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (p + t >= s0 && p + t < e0) or_into(x, ldg_lanes<W>(front, us[t]));
      }
#pragma unroll
      for (int w = 0; w < W; ++w) acc.w[w] |= warp_or64(x.w[w]);
      if (lane == 0) ex += (unsigned long long)(min(e0, base + 128) - max(s0, base));
    }
    const Lanes<W> nw = and_(acc, need);
    if (lane == 0)
#pragma unroll
      for (int w = 0; w < W; ++w)
        if (nw.w[w]) atomicOr(reinterpret_cast<unsigned long long*>(next + (int64_t)v * W + w), nw.w[w]);
  }
  if (lane != 0) ex = 0;
  ex = block_sum_u64(ex, sh);
  if (threadIdx.x == 0 && ex) atomicAdd(&c->nx_examined, ex);
}

// Bottom-up, part 3: the deferred vertices, once every chunk of their rows
// has been scanned: record the lanes found.
template <class OffT, int W>
__global__ void __launch_bounds__(kThreads) k_ms_bu_fin(MsArgs<OffT> A) {
  __shared__ unsigned long long sh[kThreads / 32];
  MsCtl* c = A.ctl;
  uint64_t* next = (c->iter & 1) ? A.fb0 : A.fb1;
  const Lanes<W> live = ctl_lanes<W>(c->live);
  const unsigned T = (unsigned)(c->iter + 1) & kIterMask;
  const int np = c->n_planes;
  const int64_t nd = c->n_def;
  MsCount<W> k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = bc_vid(A.def[i], A.n, &c->bc_site, kBcMsRecord);
    const Lanes<W> s = ld_lanes<W>(A.seen, v);
    const Lanes<W> nw = and_not(and_(ld_lanes<W>(next, v), live), s);
    st_lanes<W>(next, v, nw);
    if (!any(nw)) continue;
    const int64_t d = (int64_t)A.off[v + 1] - (int64_t)A.off[v];
    ms_found<W>(A, v, s, nw, d, T, np, k);
  }
  ms_count_flush<W>(c, k, sh, false);
}

// Writes the levels of the lanes in F.lanes (of mask word F.word) for every
// original ID, and with F.release clears those lanes' bits.
// Levels of vertex v (original ID o) for the lanes in F.lanes, with at most
// NP planes in use: the plane words are shifted right one lane at a time, so
// every lane costs a few constant-shift operations per plane.
template <int NP, int W, class OffT>
__device__ __forceinline__ void flush_vertex(const MsArgs<OffT>& A, const FlushArgs& F, int np, int64_t o, int64_t v,
                                             int32_t* const* s_out, const int32_t* s_start,
                                             unsigned long long& mu_back) {
  const int64_t vw = v * W + F.word;
  const unsigned long long s = A.seen[vw];
  const unsigned long long hit = s & F.lanes;
  unsigned long long q[NP];
#pragma unroll
  for (int b = 0; b < NP; ++b) q[b] = (hit && b < np) ? A.planes[(int64_t)b * A.n * W + vw] : 0ull;
  if (F.release && hit) {
    // a frontier bit of a lane only sits on a vertex that lane reached: clear
    // the released lanes in both frontier buffers too, so a lane reused later
    // starts from a clean frontier even if no step ran in between
    A.fb0[vw] &= ~F.lanes;
    A.fb1[vw] &= ~F.lanes;
    A.seen[vw] = s & ~F.lanes;
#pragma unroll
    for (int b = 0; b < NP; ++b)
      if (b < np) A.planes[(int64_t)b * A.n * W + vw] = q[b] & ~F.lanes;
    bool unseen = !(s & ~F.lanes);  // unseen by every lane again (the other words flush in their own launch)
#pragma unroll
    for (int w = 0; w < W; ++w)
      if (w != F.word && A.seen[v * W + w]) unseen = false;
    if (unseen) mu_back += (unsigned long long)A.firstdeg[v].y;
  }
  // lanes unrolled: every bit position is a compile-time constant, and the
  // lane test is uniform across the warp (F.lanes is the same for all threads)
#pragma unroll
  for (int i = 0; i < kMsWordLanes; ++i) {
    if (!((F.lanes >> i) & 1ull)) continue;
    int32_t lev = -1;
    if ((hit >> i) & 1ull) {
      unsigned T = 0;
#pragma unroll
      for (int b = 0; b < NP; ++b) T |= (unsigned)((q[b] >> i) & 1ull) << b;
      lev = (int32_t)((T - (unsigned)s_start[i]) & kIterMask);
    }
    s_out[i][o] = lev;
  }
}

// One kernel per plane-count class (NP = 4, 8, 16 planes at most): all three
// are launched and the ones that do not match the planes in use return at
// once, so the common case keeps a small register footprint.
template <class OffT, int W, int NP>
__global__ void __launch_bounds__(kThreads) k_ms_flush(MsArgs<OffT> A, FlushArgs F) {
  const int np = A.ctl->n_planes;
  if (np > NP || (NP > 4 && np <= NP / 2)) return;
  __shared__ int32_t* s_out[kMsWordLanes];
  __shared__ int32_t s_start[kMsWordLanes];
  if (threadIdx.x < kMsWordLanes) {
    s_out[threadIdx.x] = F.out[threadIdx.x];
    s_start[threadIdx.x] = F.start[threadIdx.x];
  }
  __syncthreads();
  unsigned long long mu_back = 0;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < A.n; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = A.o2n ? A.o2n[o] : o;
    flush_vertex<NP, W>(A, F, np, o, v, s_out, s_start, mu_back);
  }
  if (F.release) {
    __shared__ unsigned long long sh[kThreads / 32];
    mu_back = block_sum_u64(mu_back, sh);
    if (threadIdx.x == 0) {
      if (mu_back) atomicAdd(reinterpret_cast<unsigned long long*>(&A.ctl->m_u), mu_back);
      if (blockIdx.x == 0) atomicAnd(&A.ctl->active[F.word], ~F.lanes);  // the lanes are free again
    }
  }
}

// The flush for up to four discovery planes (iterations below 16, the usual
// case) with four consecutive original IDs per thread: one 16-byte map load
// and one 16-byte store per lane row instead of four of each.
template <class OffT, int W>
__global__ void __launch_bounds__(kThreads) k_ms_flush4v(MsArgs<OffT> A, FlushArgs F) {
  const int np = A.ctl->n_planes;
  if (np > 4) return;
  __shared__ int32_t* s_out[kMsWordLanes];
  __shared__ int32_t s_start[kMsWordLanes];
  if (threadIdx.x < kMsWordLanes) {
    s_out[threadIdx.x] = F.out[threadIdx.x];
    s_start[threadIdx.x] = F.start[threadIdx.x];
  }
  __syncthreads();
  unsigned long long mu_back = 0;
  const int64_t quads = A.n >> 2;
  for (int64_t qd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qd < quads; qd += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = qd * 4;
    int64_t v[4];
    if (A.o2n) {
      const int4 m4 = __ldg(reinterpret_cast<const int4*>(A.o2n) + qd);
      v[0] = m4.x;
      v[1] = m4.y;
      v[2] = m4.z;
      v[3] = m4.w;
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t) v[t] = o + t;
    }
    unsigned long long sv[4], hit[4], q[4][4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      sv[t] = A.seen[v[t] * W + F.word];
      hit[t] = sv[t] & F.lanes;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        q[t][b] = (hit[t] && b < np) ? A.planes[(int64_t)b * A.n * W + v[t] * W + F.word] : 0ull;
    if (F.release) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (!hit[t]) continue;
        const int64_t vw = v[t] * W + F.word;
        A.fb0[vw] &= ~F.lanes;
        A.fb1[vw] &= ~F.lanes;
        A.seen[vw] = sv[t] & ~F.lanes;
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (b < np) A.planes[(int64_t)b * A.n * W + vw] = q[t][b] & ~F.lanes;
        bool unseen = !(sv[t] & ~F.lanes);  // the other words flush in their own launch
#pragma unroll
        for (int w = 0; w < W; ++w)
          if (w != F.word && A.seen[v[t] * W + w]) unseen = false;
        if (unseen) mu_back += (unsigned long long)A.firstdeg[v[t]].y;
      }
    }
#pragma unroll
    for (int i = 0; i < kMsWordLanes; ++i) {
      if (!((F.lanes >> i) & 1ull)) continue;
      int32_t lev[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        unsigned T = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) T |= (unsigned)((q[t][b] >> i) & 1ull) << b;
        lev[t] = ((hit[t] >> i) & 1ull) ? (int32_t)((T - (unsigned)s_start[i]) & kIterMask) : -1;
      }
      *reinterpret_cast<int4*>(s_out[i] + o) = make_int4(lev[0], lev[1], lev[2], lev[3]);
    }
  }
  if (F.release) {
    __shared__ unsigned long long sh[kThreads / 32];
    mu_back = block_sum_u64(mu_back, sh);
    if (threadIdx.x == 0) {
      if (mu_back) atomicAdd(reinterpret_cast<unsigned long long*>(&A.ctl->m_u), mu_back);
      if (blockIdx.x == 0) atomicAnd(&A.ctl->active[F.word], ~F.lanes);
    }
  }
}

template <class OffT>
MsArgs<OffT> ms_args(MsGroup* m) {
  dobfs_graph* g = m->g;
  MsArgs<OffT> A;
  A.off = g->off.as<OffT>();
  A.cols = g->cols.as<int32_t>();
  A.firstdeg = g->firstdeg.as<int2>();
  A.o2n = g->reindexed ? g->orig2new.as<int32_t>() : nullptr;
  A.seen = m->seen.as<uint64_t>();
  A.fb0 = m->fb0.as<uint64_t>();
  A.fb1 = m->fb1.as<uint64_t>();
  A.planes = m->planes.as<uint64_t>();
  A.rec = m->rec.as<int2>();
  A.def = m->def.as<int32_t>();
  A.ctl = m->ctl.as<MsCtl>();
  A.ls = m->lstats.as<MsLaneStats>();
  A.small_tab = g->degge.as<int64_t>() + 33;
  A.small_deg = g->small_deg;
  A.n = g->n;
  A.nnz = g->nnz;
  A.n_cand = g->reindexed ? std::max<int64_t>(g->n_nonisolated, 1) : g->n;
  A.rec_cap = m->rec_cap;
  return A;
}

int ms_grid(int per_sm = 8) { return sm_count() * per_sm; }

// The main kernel of a step (top-down push or bottom-up search) with T
// threads per block, as many threads per SM as the others.
template <class OffT, int W, int NT>
void ms_main_t(const MsArgs<OffT>& A, int part, int merge, cudaStream_t s) {
  const int G = ms_grid(8 * kThreads / NT);
  if (part == 0)
    k_ms_td<OffT, W, NT><<<G, NT, 0, s>>>(A);
  else
    k_ms_bu<OffT, W, NT><<<G, NT, 0, s>>>(A, merge);
}

template <class OffT, int W>
int ms_launch_case(MsGroup* m, int kase, cudaStream_t s) {
  const MsArgs<OffT> A = ms_args<OffT>(m);
  const int G = ms_grid();
  // part 0: top-down push, 1: bottom-up search (which records the pushes too
  // in a step of both kinds)
  auto main_step = [&](int part) {
    const int t = part == 0 ? m->td_threads : m->bu_threads;
    const int merge = kase == 2 ? 1 : 0;
    if (t == 128) ms_main_t<OffT, W, 128>(A, part, merge, s);
    else if (t == 512) ms_main_t<OffT, W, 512>(A, part, merge, s);
    else ms_main_t<OffT, W, 256>(A, part, merge, s);
  };
  k_ms_clear_plane<OffT, W><<<G, kThreads, 0, s>>>(A);
  if (kase == 0) {
    k_ms_clear_next<OffT, W><<<G, kThreads, 0, s>>>(A);
    k_ms_td_list<OffT, W><<<G, kThreads, 0, s>>>(A);
    main_step(0);
    k_ms_td_post<OffT, W><<<G, kThreads, 0, s>>>(A);
  } else if (kase == 1) {
    main_step(1);
    k_ms_bu_long<OffT, W><<<G, kThreads, 0, s>>>(A);
    k_ms_bu_fin<OffT, W><<<G, kThreads, 0, s>>>(A);
  } else {  // top-down lanes pushed, then the bottom-up lanes searched and both recorded
    k_ms_clear_next<OffT, W><<<G, kThreads, 0, s>>>(A);
    k_ms_td_list<OffT, W><<<G, kThreads, 0, s>>>(A);
    main_step(0);
    k_ms_reset_records<OffT, W><<<1, 32, 0, s>>>(A);
    main_step(1);
    k_ms_bu_long<OffT, W><<<G, kThreads, 0, s>>>(A);
    k_ms_bu_fin<OffT, W><<<G, kThreads, 0, s>>>(A);
  }
  DOBFS_CUDA_TRY(cudaGetLastError());
  return DOBFS_OK;
}

template <class OffT, int W>
int ms_build_graph(MsGroup* m) {
  const MsArgs<OffT> A = ms_args<OffT>(m);
  cudaStream_t cs = nullptr;
  DOBFS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  auto fail = [&](int rc) {
    cudaStreamDestroy(cs);
    if (m->cg) cudaGraphDestroy(m->cg);
    m->cg = nullptr;
    return rc;
  };
  if (cudaGraphCreate(&m->cg, 0) != cudaSuccess) return fail(set_error(DOBFS_ERR_CUDA, "cudaGraphCreate failed"));
  cudaGraphConditionalHandle h_while, h_case;
  if (cudaGraphConditionalHandleCreate(&h_while, m->cg, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return fail(set_error(DOBFS_ERR_CUDA, "conditional handle failed"));
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = h_while;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  if (cudaGraphAddNode(&wnode, m->cg, nullptr, nullptr, 0, &wp) != cudaSuccess)
    return fail(set_error(DOBFS_ERR_CUDA, "while node failed"));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  if (cudaGraphConditionalHandleCreate(&h_case, body, 0, 0) != cudaSuccess)
    return fail(set_error(DOBFS_ERR_CUDA, "conditional handle failed"));
  if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return fail(set_error(DOBFS_ERR_CUDA, "capture failed"));
  k_ms_lane_stats<OffT, W><<<ms_grid(1), kThreads, 0, cs>>>(A);
  k_ms_switch<OffT, W><<<1, 32, 0, cs>>>(A, h_while, h_case, 1);
  cudaGraph_t captured = nullptr;
  if (cudaStreamEndCapture(cs, &captured) != cudaSuccess) return fail(set_error(DOBFS_ERR_CUDA, "end capture failed"));
  // the switch node (the one without a successor) is followed by the step's switch node
  size_t nn = 0;
  cudaGraphGetNodes(body, nullptr, &nn);
  if (nn != 2) return fail(set_error(DOBFS_ERR_CUDA, "unexpected body node count %zu", nn));
  cudaGraphNode_t bn[2];
  cudaGraphGetNodes(body, bn, &nn);
  cudaGraphNode_t sw = bn[1];
  for (int i = 0; i < 2; ++i) {
    size_t ndep = 0;
    cudaGraphNodeGetDependentNodes(bn[i], nullptr, nullptr, &ndep);
    if (ndep == 0) sw = bn[i];
  }
  cudaGraphNodeParams sp = {};
  sp.type = cudaGraphNodeTypeConditional;
  sp.conditional.handle = h_case;
  sp.conditional.type = cudaGraphCondTypeSwitch;
  sp.conditional.size = kMsCases;
  cudaGraphNode_t snode;
  if (cudaGraphAddNode(&snode, body, &sw, nullptr, 1, &sp) != cudaSuccess)
    return fail(set_error(DOBFS_ERR_CUDA, "switch node failed"));
  for (int k = 0; k < kMsCases; ++k) {
    if (cudaStreamBeginCaptureToGraph(cs, sp.conditional.phGraph_out[k], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return fail(set_error(DOBFS_ERR_CUDA, "capture case failed"));
    const int rc = ms_launch_case<OffT, W>(m, k, cs);
    cudaGraph_t cap = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &cap);
    if (rc != DOBFS_OK) return fail(rc);
    if (e != cudaSuccess) return fail(set_error(DOBFS_ERR_CUDA, "end capture case: %s", cudaGetErrorString(e)));
  }
  const cudaError_t e = cudaGraphInstantiate(&m->exec, m->cg, 0);
  if (e != cudaSuccess) return fail(set_error(DOBFS_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e)));
  cudaStreamDestroy(cs);
  m->graph_bu = m->bu_threads;
  m->graph_td = m->td_threads;
  return DOBFS_OK;
}

template <class OffT, int W>
int ms_seed_impl(MsGroup* m, const SeedArgs& S) {
  k_ms_seed<OffT, W><<<1, kMsLanes, 0, m->stream>>>(ms_args<OffT>(m), S);
  DOBFS_CUDA_TRY(cudaGetLastError());
  return DOBFS_OK;
}

template <class OffT, int W>
int ms_step_impl(MsGroup* m, MsCtl* after_switch, float* case_ms) {
  const MsArgs<OffT> A = ms_args<OffT>(m);
  k_ms_lane_stats<OffT, W><<<ms_grid(1), kThreads, 0, m->stream>>>(A);
  k_ms_switch<OffT, W><<<1, 32, 0, m->stream>>>(A, 0, 0, 0);
  MsCtl c;
  DOBFS_CUDA_TRY(cudaMemcpyAsync(&c, m->ctl.ptr, sizeof(c), cudaMemcpyDeviceToHost, m->stream));
  DOBFS_CUDA_TRY(cudaStreamSynchronize(m->stream));
  if (after_switch) *after_switch = c;
  if (c.done) return DOBFS_OK;  // no live lane
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (case_ms) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, m->stream);
  }
  const int rc = ms_launch_case<OffT, W>(m, c.step_case, m->stream);
  if (case_ms) {
    cudaEventRecord(e1, m->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(case_ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  return rc;
}

template <class OffT, int W>
int ms_flush_impl(MsGroup* m, const FlushArgs& F) {
  const int G = (int)std::min<int64_t>(ceil_div(m->g->n, kThreads), (int64_t)ms_grid(16));
  const MsArgs<OffT> A = ms_args<OffT>(m);
  if (F.vec)
    k_ms_flush4v<OffT, W><<<G, kThreads, 0, m->stream>>>(A, F);
  else
    k_ms_flush<OffT, W, 4><<<G, kThreads, 0, m->stream>>>(A, F);
  k_ms_flush<OffT, W, 8><<<G, kThreads, 0, m->stream>>>(A, F);
  k_ms_flush<OffT, W, 16><<<G, kThreads, 0, m->stream>>>(A, F);
  DOBFS_CUDA_TRY(cudaGetLastError());
  return DOBFS_OK;
}

template <class OffT, int W>
int ms_switch_async_impl(MsGroup* m, MsCtl* dst) {
  k_ms_lane_stats<OffT, W><<<ms_grid(1), kThreads, 0, m->stream>>>(ms_args<OffT>(m));
  k_ms_switch<OffT, W><<<1, 32, 0, m->stream>>>(ms_args<OffT>(m), 0, 0, 0);
  DOBFS_CUDA_TRY(cudaGetLastError());
  DOBFS_CUDA_TRY(cudaMemcpyAsync(dst, m->ctl.ptr, sizeof(MsCtl), cudaMemcpyDeviceToHost, m->stream));
  return DOBFS_OK;
}

template <class OffT, int W>
int ms_rebase_impl(MsGroup* m) {
  k_ms_rebase<OffT, W><<<1, 32, 0, m->stream>>>(ms_args<OffT>(m));
  DOBFS_CUDA_TRY(cudaGetLastError());
  return DOBFS_OK;
}

// Calls F<OffT, W>(args...) for the group's offset type and mask words.
#define MS_DISPATCH(m, F, ...)                                                            \
  ((m)->g->off64 ? ((m)->words == 2 ? F<int64_t, 2>(__VA_ARGS__) : F<int64_t, 1>(__VA_ARGS__)) \
                 : ((m)->words == 2 ? F<int32_t, 2>(__VA_ARGS__) : F<int32_t, 1>(__VA_ARGS__)))

}  // namespace

int ms_group_switch_async(MsGroup* m, MsCtl* dst) { return MS_DISPATCH(m, ms_switch_async_impl, m, dst); }

int ms_group_case_async(MsGroup* m, int kase) { return MS_DISPATCH(m, ms_launch_case, m, kase, m->stream); }

int64_t ms_group_bytes(const dobfs_graph* g, int words) {
  const int64_t n_cand = g->reindexed ? std::max<int64_t>(g->n_nonisolated, 1) : g->n;
  return (int64_t)sizeof(uint64_t) * g->n * words * (3 + kMsPlanes) +
         (int64_t)sizeof(int2) * (n_cand + g->nnz / kMsChunkMin + 64) + (int64_t)sizeof(int32_t) * g->n +
         (int64_t)sizeof(MsCtl) + (int64_t)sizeof(MsLaneStats);
}

int ms_group_create(dobfs_graph* g, cudaStream_t s, int words, MsGroup** out) {
  if (words < 1 || words > kMsMaxWords) return set_error(DOBFS_ERR_INVALID, "lane groups hold 1 or 2 mask words");
  MsGroup* m = new (std::nothrow) MsGroup();
  if (!m) return set_error(DOBFS_ERR_OOM, "host allocation failed");
  m->g = g;
  m->stream = s;
  m->words = words;
  const size_t vb = sizeof(uint64_t) * (size_t)g->n * (size_t)words;
  int rc = m->seen.alloc(vb, s);
  if (rc == DOBFS_OK) rc = m->fb0.alloc(vb, s);
  if (rc == DOBFS_OK) rc = m->fb1.alloc(vb, s);
  if (rc == DOBFS_OK) rc = m->planes.alloc(vb * kMsPlanes, s);
  const int64_t n_cand = g->reindexed ? std::max<int64_t>(g->n_nonisolated, 1) : g->n;
  m->rec_cap = n_cand + g->nnz / kMsChunkMin + 64;
  if (rc == DOBFS_OK) rc = m->rec.alloc(sizeof(int2) * (size_t)m->rec_cap, s);
  if (rc == DOBFS_OK) rc = m->def.alloc(sizeof(int32_t) * (size_t)g->n, s);
  if (rc == DOBFS_OK) rc = m->ctl.alloc(sizeof(MsCtl), s);
  if (rc == DOBFS_OK) rc = m->lstats.alloc(sizeof(MsLaneStats), s);
  if (rc != DOBFS_OK) {
    delete m;
    return rc;
  }
  *out = m;
  return DOBFS_OK;
}

void ms_group_destroy(MsGroup* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  if (m->exec) cudaGraphExecDestroy(m->exec);
  if (m->cg) cudaGraphDestroy(m->cg);
  delete m;
}

int ms_group_reset(MsGroup* m, const dobfs_run_opts& o) {
  cudaStream_t s = m->stream;
  const size_t vb = sizeof(uint64_t) * (size_t)m->g->n * (size_t)m->words;
  DOBFS_CUDA_TRY(cudaMemsetAsync(m->seen.ptr, 0, vb, s));
  DOBFS_CUDA_TRY(cudaMemsetAsync(m->fb0.ptr, 0, vb, s));
  DOBFS_CUDA_TRY(cudaMemsetAsync(m->fb1.ptr, 0, vb, s));
  // iterations below 16 need kFirstPlanes planes; later planes are cleared on first use
  DOBFS_CUDA_TRY(cudaMemsetAsync(m->planes.ptr, 0, vb * kFirstPlanes, s));
  DOBFS_CUDA_TRY(cudaMemsetAsync(m->lstats.ptr, 0, sizeof(MsLaneStats), s));
  MsCtl c;
  memset(&c, 0, sizeof(c));
  c.fresh = 1;
  c.n_planes = kFirstPlanes;
  c.clear_plane = -1;
  c.m_u = m->g->nnz;
  c.mode = o.direction;
  c.alpha = o.alpha;
  c.beta = o.beta;
  c.td_chunk = o.td_chunk ? o.td_chunk : kMsChunk;
  c.bu_scan = o.bu_scan ? o.bu_scan : kMsT;
  c.sched_seed = o.schedule_seed;
  m->bu_threads = o.bu_threads ? o.bu_threads : kThreads;
  m->td_threads = o.td_threads ? o.td_threads : kThreads;
  // written by a kernel that takes the block by value, so the host neither
  // keeps a staging copy alive nor waits for the stream
  k_ms_set_ctl<<<1, 1, 0, s>>>(m->ctl.as<MsCtl>(), c);
  DOBFS_CUDA_TRY(cudaGetLastError());
  return DOBFS_OK;
}

int ms_group_seed(MsGroup* m, int count, const int32_t* lane, const int32_t* root) {
  if (count < 0 || count > kMsWordLanes * m->words) return set_error(DOBFS_ERR_INVALID, "more lanes than the group has");
  SeedArgs S;
  S.count = count;
  for (int i = 0; i < count; ++i) {
    if (lane[i] < 0 || lane[i] >= kMsWordLanes * m->words) return set_error(DOBFS_ERR_INVALID, "lane out of range");
    S.lane[i] = lane[i];
    S.root[i] = root[i];
  }
  return MS_DISPATCH(m, ms_seed_impl, m, S);
}

int ms_group_step(MsGroup* m, MsCtl* after_switch, float* case_ms) {
  return MS_DISPATCH(m, ms_step_impl, m, after_switch, case_ms);
}

int ms_group_run_to_end(MsGroup* m) {
  if (m->exec && (m->graph_bu != m->bu_threads || m->graph_td != m->td_threads)) {
    // the loop graph was built for other block sizes: rebuild it (the
    // group's stream orders it after any launch still running)
    DOBFS_CUDA_TRY(cudaStreamSynchronize(m->stream));
    cudaGraphExecDestroy(m->exec);
    cudaGraphDestroy(m->cg);
    m->exec = nullptr;
    m->cg = nullptr;
  }
  if (!m->exec) DOBFS_TRY(MS_DISPATCH(m, ms_build_graph, m));
  DOBFS_CUDA_TRY(cudaGraphLaunch(m->exec, m->stream));
  return DOBFS_OK;
}

int ms_group_flush(MsGroup* m, LaneMask lanes, int32_t* const* out, const int32_t* start, bool release) {
  for (int w = 0; w < m->words; ++w) {
    const uint64_t lw = lane_word(lanes, w);
    if (!lw) continue;
    FlushArgs F;
    memset(&F, 0, sizeof(F));
    F.lanes = lw;
    F.word = w;
    F.release = release ? 1 : 0;
    F.vec = (m->g->n % 4 == 0) ? 1 : 0;
    for (int i = 0; i < kMsWordLanes; ++i) {
      const int l = kMsWordLanes * w + i;
      F.out[i] = ((lw >> i) & 1ull) ? out[l] : nullptr;
      F.start[i] = start ? start[l] : 0;
      if (F.out[i] && (reinterpret_cast<uintptr_t>(F.out[i]) & 15)) F.vec = 0;
    }
    DOBFS_TRY(MS_DISPATCH(m, ms_flush_impl, m, F));
  }
  return DOBFS_OK;
}

int ms_group_rebase(MsGroup* m) { return MS_DISPATCH(m, ms_rebase_impl, m); }

int ms_group_read_ctl(MsGroup* m, MsCtl* c) {
  DOBFS_CUDA_TRY(cudaMemcpyAsync(c, m->ctl.ptr, sizeof(MsCtl), cudaMemcpyDeviceToHost, m->stream));
  DOBFS_CUDA_TRY(cudaStreamSynchronize(m->stream));
  return DOBFS_OK;
}

}  // namespace dobfs

using namespace dobfs;

extern "C" int dobfs_run_batch(dobfs_graph* g, const int32_t* roots, int32_t n_roots, int32_t* level_out,
                               int32_t* parent_out, const dobfs_run_opts* opts, dobfs_run_stats* stats) {
  clear_error();
  if (!g || n_roots < 0 || (n_roots > 0 && (!roots || !level_out)))
    return set_error(DOBFS_ERR_INVALID, "graph, roots and level_out are required");
  if (parent_out)
    return set_error(DOBFS_ERR_INVALID,
                     "dobfs_run_batch produces levels only; use dobfs_run for parents (parent_out must be NULL)");
  dobfs_run_opts o;
  dobfs_run_opts_init(&o);
  o.alpha = DOBFS_BATCH_ALPHA;
  if (opts) o = *opts;
  if (o.direction < 0 || o.direction > DOBFS_DIR_RANDOM || o.alpha < 1 || o.beta < 1)
    return set_error(DOBFS_ERR_INVALID, "bad run options for a batch (direction must be auto, top-down, "
                                        "bottom-up or random)");
  if (!cutoffs_valid(o)) return set_error(DOBFS_ERR_INVALID, "bad degree-bin cutoffs");
  if (n_roots == 0) {  // nothing to run (roots and level_out may be NULL)
    if (stats) memset(stats, 0, sizeof(*stats));
    return DOBFS_OK;
  }
  std::vector<int32_t> hroots((size_t)n_roots);
  if (n_roots > 0) {
    if (is_device_ptr(roots))
      DOBFS_CUDA_TRY(cudaMemcpy(hroots.data(), roots, sizeof(int32_t) * (size_t)n_roots, cudaMemcpyDeviceToHost));
    else
      memcpy(hroots.data(), roots, sizeof(int32_t) * (size_t)n_roots);
  }
  for (int32_t i = 0; i < n_roots; ++i)
    if (hroots[i] < 0 || hroots[i] >= g->n)
      return set_error(DOBFS_ERR_INVALID, "root %d (index %d) out of range [0, %lld)", hroots[i], i, (long long)g->n);
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t s = o.stream ? (cudaStream_t)o.stream : g->stream;
  if (g->last_stream && g->last_stream != s) DOBFS_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_done, 0));
  // more than 64 roots run in 128-lane groups: a wide bottom-up step costs
  // about the same for 128 lanes as for 64
  const int words = n_roots > kMsWordLanes ? 2 : 1;
  const int group_lanes = kMsWordLanes * words;
  if (g->ms && g->ms->words != words) {
    ms_group_destroy(g->ms);
    g->ms = nullptr;
  }
  if (!g->ms) DOBFS_TRY(ms_group_create(g, s, words, &g->ms));
  const bool dev_out = is_device_ptr(level_out);
  const size_t stage_bytes = sizeof(int32_t) * (size_t)group_lanes * (size_t)g->n;
  if (!dev_out && g->ms_stage.bytes < stage_bytes) DOBFS_TRY(g->ms_stage.alloc(stage_bytes, g->stream));
  const bool host_loop = (o.flags & DOBFS_RUN_HOST_LOOP) != 0;
  // Batches of several groups with device outputs run up to kMsConcurrent
  // groups at a time, each on its own stream, the groups taken in turn:
  // one group's latency-bound steps overlap another's bandwidth-bound flush.
  // A further group is created only while the device keeps at least one
  // more group's worth of memory free after it (else fewer run at a time);
  // with statistics, host outputs, host-driven levels or bounds checks,
  // which read each group back in turn, the groups run one after another.
  const int n_groups = (int)ceil_div(n_roots, group_lanes);
  int par = (dev_out && !host_loop && !stats && !kBoundsCheck) ? std::min(n_groups, kMsConcurrent) : 1;
  for (int k = 0; k + 1 < par; ++k) {
    if (g->ms_more[k] && g->ms_more[k]->words != words) {
      ms_group_destroy(g->ms_more[k]);
      g->ms_more[k] = nullptr;
    }
    bool ok = true;
    if (!g->ms_streams[k])
      ok = cudaStreamCreateWithFlags(&g->ms_streams[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&g->ms_ev_join[k], cudaEventDisableTiming) == cudaSuccess;
    if (ok && !g->ms_ev_fork) ok = cudaEventCreateWithFlags(&g->ms_ev_fork, cudaEventDisableTiming) == cudaSuccess;
    if (ok && !g->ms_more[k]) {
      size_t free_b = 0, total_b = 0;
      ok = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && (int64_t)free_b >= 2 * ms_group_bytes(g, words) &&
           ms_group_create(g, g->ms_streams[k], words, &g->ms_more[k]) == DOBFS_OK;
    }
    if (!ok) {  // no memory (or stream) for this group: fewer groups at a time
      cudaGetLastError();
      clear_error();
      par = k + 1;
      break;
    }
  }
  g->batch_trace.clear();
  g->last_trace_batch = host_loop;
  DOBFS_CUDA_TRY(cudaEventRecord(g->ev_t0, s));
  if (par > 1) {  // the other streams start after everything queued on s so far
    DOBFS_CUDA_TRY(cudaEventRecord(g->ms_ev_fork, s));
    for (int k = 0; k + 1 < par; ++k) DOBFS_CUDA_TRY(cudaStreamWaitEvent(g->ms_streams[k], g->ms_ev_fork, 0));
  }
  int32_t max_levels = 0;
  int64_t examined = 0, alg_bytes = 0;
  for (int32_t b0 = 0; b0 < n_roots; b0 += group_lanes) {
    const int cnt = (int)std::min<int32_t>(group_lanes, n_roots - b0);
    const int slot = (b0 / group_lanes) % par;
    MsGroup* m = slot ? g->ms_more[slot - 1] : g->ms;
    m->stream = slot ? g->ms_streams[slot - 1] : s;
    DOBFS_TRY(ms_group_reset(m, o));
    int32_t lanes[kMsLanes];
    for (int i = 0; i < cnt; ++i) lanes[i] = i;
    DOBFS_TRY(ms_group_seed(m, cnt, lanes, hroots.data() + b0));
    if (host_loop) {
      // host-driven levels, each timed (diagnostics); the trace keeps the first group
      for (int guard = 0; guard < (1 << 16) + 2; ++guard) {
        MsCtl c;
        float ms_case = 0.f;
        DOBFS_TRY(ms_group_step(m, &c, &ms_case));
        if (c.done) break;
        if (b0 == 0) {
          dobfs_level_trace t;
          memset(&t, 0, sizeof(t));
          t.level = c.levels_run;
          t.direction = c.dir;
          t.n_frontier = c.n_f;
          t.m_frontier = c.m_f;
          t.m_unvisited = c.m_u;
          t.edges_examined = c.examined;  // running total; differenced below
          t.ms = ms_case;
          t.ms_main = ms_case;
          g->batch_trace.push_back(t);
        }
      }
      if (b0 == 0 && !g->batch_trace.empty()) {
        // edges_examined holds running totals taken before each step: turn them into per-step counts
        MsCtl fin;
        DOBFS_TRY(ms_group_read_ctl(m, &fin));
        for (size_t i = 0; i < g->batch_trace.size(); ++i) {
          const int64_t next_total = (i + 1 < g->batch_trace.size()) ? g->batch_trace[i + 1].edges_examined : fin.examined;
          g->batch_trace[i].vertices_scanned = next_total;  // scratch
        }
        for (size_t i = 0; i < g->batch_trace.size(); ++i) {
          g->batch_trace[i].edges_examined = g->batch_trace[i].vertices_scanned - g->batch_trace[i].edges_examined;
          g->batch_trace[i].vertices_scanned = 0;
        }
      }
    } else {
      DOBFS_TRY(ms_group_run_to_end(m));
    }
    int32_t* outp[kMsLanes];
    for (int i = 0; i < kMsLanes; ++i)
      outp[i] = i < cnt ? (dev_out ? level_out + (int64_t)(b0 + i) * g->n : g->ms_stage.as<int32_t>() + (int64_t)i * g->n)
                        : nullptr;
    const LaneMask lm = cnt == kMsLanes ? ~(LaneMask)0 : (lane_bit(cnt) - 1);
    DOBFS_TRY(ms_group_flush(m, lm, outp, nullptr, false));
    if (!dev_out)
      DOBFS_CUDA_TRY(cudaMemcpyAsync(level_out + (int64_t)b0 * g->n, g->ms_stage.ptr,
                                     sizeof(int32_t) * (size_t)cnt * (size_t)g->n, cudaMemcpyDeviceToHost, s));
    if (stats || kBoundsCheck) {
      MsCtl c;
      DOBFS_TRY(ms_group_read_ctl(m, &c));
      if (c.bc_site)
        return set_error(DOBFS_ERR_BOUNDS, "device bounds check failed: %s", bounds_site_name(c.bc_site));
      if (c.runaway) return set_error(DOBFS_ERR_CUDA, "internal: the batch loop ran past n iterations");
      max_levels = std::max(max_levels, c.levels_run);
      examined += c.examined;
      // the steps' bytes, plus the flush: one 4-byte level per (vertex, lane)
      alg_bytes += c.alg_bytes + 4 * (int64_t)cnt * g->n;
    }
  }
  for (int k = 0; k + 1 < par; ++k) {  // s waits for the other streams' groups
    DOBFS_CUDA_TRY(cudaEventRecord(g->ms_ev_join[k], g->ms_streams[k]));
    DOBFS_CUDA_TRY(cudaStreamWaitEvent(s, g->ms_ev_join[k], 0));
  }
  DOBFS_CUDA_TRY(cudaEventRecord(g->ev_t1, s));
  DOBFS_CUDA_TRY(cudaEventRecord(g->ev_done, s));
  g->last_stream = s;
  if (!dev_out || stats) DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev_t0, g->ev_t1);
    stats->device_ms = ms;
    stats->levels = max_levels;
    stats->edges_examined = examined;
    stats->alg_bytes = alg_bytes;
  }
  return DOBFS_OK;
}
