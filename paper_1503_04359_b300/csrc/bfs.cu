// Direction-optimized BFS on one GPU: the per-level step of Algorithm 1 with
// the direction switch of Sec. 3.3, all on the device.
//
// State in HBM (internal vertex IDs):
//   visited  bitmap, one bit per vertex (the isVisited flag of Algorithm 1)
//   fbm[2]   frontier bitmaps, level parity selects current / next
//   q[2]     frontier queues (int32), level parity selects current / next
//   lp       int2 per vertex: (level, parent), written once when discovered
//   ctl      BfsCtl: frontier counts n_f, m_f, unvisited edge count m_u, ...
//
// One level = one "step":
//   top-down  (Algorithm 1, top-down branch): every frontier vertex reads its
//             row and claims unvisited neighbours with atomicOr on the visited
//             bitmap; the winner writes (level, parent) and appends the vertex
//             to the next queue. Rows of up to td_small_max entries are expanded
//             by one thread in the binning kernel; longer rows are cut into
//             td_chunk-entry records expanded one warp each with 16-byte loads.
//   bottom-up (Algorithm 1, bottom-up branch): a warp owns one visited-bitmap
//             word (32 consecutive vertices); each unvisited vertex scans its
//             row in order and stops at the first neighbour whose frontier
//             bit is set. The warp writes the next-frontier word and the
//             visited word with one store each (ballot), no atomics. Rows
//             with no hit among their first bu_scan entries continue in a
//             warp-per-row kernel (16-byte loads, ballot for the first hit).
//   switch    (Sec. 3.3): a one-thread kernel folds the step's counters into
//             n_f, m_f, m_u and picks the next direction: top-down -> bottom-up
//             when m_f * alpha > m_u, bottom-up -> top-down when the frontier
//             shrinks below n / beta (the alpha/beta rule of the direction-
//             optimizing BFS the paper builds on), or the paper's own static
//             policy. Conversions (queue -> bitmap, bitmap -> queue) run only
//             when the direction changes.
// The level loop is a CUDA graph: a while node whose body is the switch
// kernel followed by a switch node over the four step kinds, so the host
// launches one graph per BFS and never waits between levels.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "../../dobfs_inputs/gen.h"
#include "common.cuh"
#include "graph.cuh"
#include "msbfs.cuh"

namespace cg = cooperative_groups;

namespace dobfs {

namespace {

constexpr int kThreads = 256;
// Degree-bin cutoffs (defaults; a run may set others, read from BfsCtl):
constexpr int kTdSmall = 16;     // top-down rows up to this length: one thread
constexpr int kChunk = 512;      // top-down chunk record length (entries)
constexpr int kBuT = 32;         // bottom-up entries scanned per thread before deferring
constexpr int kTdClaimPer = 8;   // top-down chunk entries claimed per lane per step (4: 0.5 % slower at scale 28)
constexpr int kTdSmallMin = 8;   // smallest allowed cutoffs (they size the record buffer)
constexpr int kChunkMin = 256;
constexpr int kCases = 6;      // step kinds of the level loop's switch node
// Threads per block of the step kernels a run may choose (block sizes change
// only the speed, never the result): 128, 256 (default) or 512.
__host__ __device__ constexpr int bu_min_blocks(int t) { return t <= 128 ? 10 : (t <= 256 ? 5 : 2); }
constexpr int kCaseNone = 7;   // switch value with no body: loop ends

template <class OffT>
struct BfsArgs {
  const OffT* off;
  const int32_t* cols;
  const uint32_t* iso;
  const int32_t* o2n;  // NULL when not reindexed
  const int2* firstdeg;  // (first neighbour, degree) per vertex; first = -1 for isolated vertices
  const int64_t* deg_ge;  // [33]: vertices of degree >= 2^k
  const int64_t* small_tab;  // [2 * kSmallDeg]: row offset and first ID of each small degree (renumbered graphs)
  int32_t small_deg;         // degrees below this use small_tab for the row start (0: none)
  uint32_t* visited;
  uint32_t* fbm0;
  uint32_t* fbm1;
  int2* lp;
  int32_t* q0;
  int32_t* q1;
  int2* rec;
  int32_t* def;
  BfsCtl* ctl;
  uint32_t* gbar;  // grid barrier of the fused loop: arrivals, generation, timed-out flag
  LevelRec* trace;
  int64_t n, nnz, words, cand_words, rec_cap, n_nonisolated;
};

// Loads of data that the level loop writes (bitmaps, queues, records,
// deferred rows). In the separate kernels of the graph-driven loop such data
// does not change while a kernel runs, so it is read through the read-only
// or L1 path. The fused loop for small graphs (COH) runs every level in one
// kernel: there another SM may have written the data since this SM last
// cached it, so it is read from L2 (coherent).
template <bool COH, class T>
__device__ __forceinline__ T ld_mut(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}
template <bool COH>
__device__ __forceinline__ uint32_t ld_ro(const uint32_t* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}

template <bool COH = false>
__device__ __forceinline__ bool test_bit(const uint32_t* __restrict__ bm, int32_t v) {
  return (ld_ro<COH>(bm + (v >> 5)) >> (v & 31)) & 1u;
}

// First position in the sorted row cols[s, e) whose column is >= x.
__device__ __forceinline__ int64_t lower_bound_col(const int32_t* __restrict__ cols, int64_t s, int64_t e, int32_t x) {
  while (s < e) {
    const int64_t m = s + ((e - s) >> 1);
    if (__ldg(cols + m) < x) s = m + 1; else e = m;
  }
  return s;
}

// Appends v to q at an index taken from *tail, one atomic per group of
// converged threads.
__device__ __forceinline__ void enqueue(unsigned int* tail, int32_t* q, int32_t v, int64_t cap, int32_t* bc,
                                        int site) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(tail, g.size());
  base = g.shfl(base, 0);
  if (bc_pos((int64_t)base + g.thread_rank(), cap, bc, site)) q[base + g.thread_rank()] = v;
}

// Four top-down claims at once: the visited words are read first, then the
// atomics for the still-unvisited neighbours are issued together, then the
// winners write (level, parent) and read their degree. Keeping the four
// chains independent overlaps their memory latencies. Returns the winners
// as a 4-bit mask; `m_new` accumulates their degrees.
template <int N, class OffT>
__device__ __forceinline__ unsigned td_claimN(const BfsArgs<OffT>& A, const int32_t (&v)[N], unsigned valid,
                                              int32_t u, int32_t next_level, unsigned long long& m_new) {
  uint32_t w[N];
#pragma unroll
  for (int t = 0; t < N; ++t) w[t] = ((valid >> t) & 1u) ? __ldcg(A.visited + (v[t] >> 5)) : ~0u;
  unsigned cand = 0;
#pragma unroll
  for (int t = 0; t < N; ++t)
    if (!((w[t] >> (v[t] & 31)) & 1u)) cand |= 1u << t;
  unsigned won = 0;
#pragma unroll
  for (int t = 0; t < N; ++t)
    if ((cand >> t) & 1u) {
      const uint32_t bit = 1u << (v[t] & 31);
      if (!(atomicOr(A.visited + (v[t] >> 5), bit) & bit)) won |= 1u << t;
    }
  int32_t d[N];
#pragma unroll
  for (int t = 0; t < N; ++t) {
    d[t] = 0;
    if ((won >> t) & 1u) {
      A.lp[v[t]] = make_int2(next_level, u);
      d[t] = __ldg(&A.firstdeg[v[t]].y);
    }
  }
#pragma unroll
  for (int t = 0; t < N; ++t) m_new += (unsigned long long)d[t];
  return won;
}

template <class OffT>
__device__ __forceinline__ unsigned td_claim4(const BfsArgs<OffT>& A, const int32_t (&v)[4], unsigned valid,
                                              int32_t u, int32_t next_level, unsigned long long& m_new) {
  return td_claimN<4>(A, v, valid, u, next_level, m_new);
}

// Top-down marking without claims (bitmap-output top-down steps): a
// neighbour not yet visited gets its bit in the next-frontier bitmap. The
// visited bitmap is read-only during the marking, so it is read through the
// read-only cache; a bit already set in the next bitmap needs no atomic.
// Parents are recovered afterwards from the frontier bitmap (k_bu in
// recovery mode).
template <bool COH, class OffT>
__device__ __forceinline__ void td_mark4(const BfsArgs<OffT>& A, const int32_t (&v)[4], unsigned valid,
                                         uint32_t* next) {
  uint32_t w[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) w[t] = ((valid >> t) & 1u) ? ld_ro<COH>(A.visited + (v[t] >> 5)) : ~0u;
  uint32_t nw[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) nw[t] = ((w[t] >> (v[t] & 31)) & 1u) ? ~0u : __ldcg(next + (v[t] >> 5));
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const uint32_t bit = 1u << (v[t] & 31);
    if (!(nw[t] & bit)) atomicOr(next + (v[t] >> 5), bit);
  }
}

// Run parameters the status init writes into the control block.
struct RunParams {
  int32_t root_orig, mode, alpha, beta, static_pct, bu_steps, td_bm_div, td_small, td_chunk, bu_scan, td_split_pct;
  uint64_t sched_seed;
};

// Status init (one thread): the control block and the root.
template <class OffT>
__device__ void init_body(const BfsArgs<OffT>& A, const RunParams& P) {
  const int32_t root_orig = P.root_orig, mode = P.mode, alpha = P.alpha, beta = P.beta;
  const int32_t static_pct = P.static_pct, bu_steps = P.bu_steps, td_bm_div = P.td_bm_div;
  const int32_t td_small = P.td_small, td_chunk = P.td_chunk, bu_scan = P.bu_scan, td_split_pct = P.td_split_pct;
  const uint64_t sched_seed = P.sched_seed;
  const int32_t r = A.o2n ? A.o2n[root_orig] : root_orig;
  const int64_t d = (int64_t)A.off[r + 1] - (int64_t)A.off[r];
  BfsCtl* c = A.ctl;
  c->level = 0;
  c->dir = 0;
  c->fmt = 0;
  c->step_case = 0;
  c->fresh = 1;
  c->done = 0;
  c->bu_run = 0;
  c->n_levels = 0;
  c->n_f = 1;
  c->m_f = d;
  c->n_f_prev = 0;
  c->m_u = A.nnz - d;
  c->nx_n = c->nx_m = c->nx_examined = c->nx_scanned = 0;
  c->q_tail = c->n_rec = c->n_def = c->conv_tail = 0;
  c->out_next = 0;
  c->reached = 1;
  c->teps2 = d;
  c->examined = 0;
  c->alg_bytes = 0;
  c->n_td = c->n_bu = 0;
  c->overflow = 0;
  c->bc_site = 0;
  c->mode = mode;
  c->alpha = alpha;
  c->beta = beta;
  c->static_pct = static_pct;
  c->bu_steps = bu_steps;
  c->sched_seed = sched_seed;
  c->td_bm_div = td_bm_div;
  c->td_small = td_small;
  c->td_chunk = td_chunk;
  c->bu_scan = bu_scan;
  c->td_split_pct = td_split_pct;
  c->split_w = 0;
  A.q0[0] = r;
  atomicOr(A.visited + (r >> 5), 1u << (r & 31));
  A.lp[r] = make_int2(0, r);
}

template <class OffT>
__global__ void k_init(BfsArgs<OffT> A, RunParams P) {
  if (threadIdx.x == 0 && blockIdx.x == 0) init_body(A, P);
}

// The direction switch (one thread): closes the step that just ran, then
// picks the next. Returns the step kind, or kCaseNone when the loop ends.
template <class OffT>
__device__ __forceinline__ int switch_decide(const BfsArgs<OffT>& A, BfsCtl* c) {
  if (!c->fresh) {
    const int32_t L = c->level;
    // top-down steps with queue output count their new vertices in the queue
    const bool queue_out = (c->step_case == 0 || c->step_case == 2);
    const int64_t n_new = queue_out ? (int64_t)c->q_tail : (int64_t)c->nx_n;
    const int64_t m_new = (int64_t)c->nx_m;
    const int64_t ex = (int64_t)c->nx_examined, sc = (int64_t)c->nx_scanned;
    int64_t bytes;
    if (c->step_case >= 4)  // bitmap-output top-down (+ bottom-up part of a mixed level, + parent search):
      // queue 4 and row bounds 16 per frontier vertex, columns 4 each read, row bounds 8 per vertex
      // searched bottom-up, level+parent 8 and bitmap conversion 4 per new vertex, conversion 4 per frontier vertex
      bytes = 24 * c->n_f + 4 * ex + 8 * sc + 12 * n_new;
    else if (c->dir == 0)  // queue read 4, row bounds 16, columns 4 each, level+parent 8 and enqueue 4 per new vertex
      bytes = 20 * c->n_f + 4 * c->m_f + 12 * n_new + (c->step_case >= 2 ? 4 * c->n_f : 0);
    else  // row bounds 8 per scanned vertex, columns 4 each read, level+parent 8 per new vertex
      bytes = 8 * sc + 4 * ex + 8 * n_new + (c->step_case == 3 ? 4 * c->n_f : 0);
    if (L < kMaxTrace) {
      LevelRec& t = A.trace[L];
      t.level = L;
      t.dir = (c->dir == 0 && c->split_w > 0) ? 2 : c->dir;
      t.n_f = c->n_f;
      t.m_f = c->m_f;
      t.m_u = c->m_u;
      t.n_next = n_new;
      t.examined = ex;
      t.scanned = sc;
      t.bytes = bytes;
    }
    c->alg_bytes += bytes;
    c->examined += ex;
    if (c->dir == 0) c->n_td += 1; else c->n_bu += 1;
    c->m_u -= m_new;
    c->teps2 += m_new;
    c->reached += n_new;
    c->n_f_prev = c->n_f;
    c->n_f = n_new;
    c->m_f = m_new;
    c->level = L + 1;
    c->fmt = queue_out ? 0 : 1;  // queue-output top-down leaves a queue, the other steps a bitmap
    c->bu_run = (c->dir == 1) ? c->bu_run + 1 : 0;
    c->nx_n = c->nx_m = c->nx_examined = c->nx_scanned = 0;
    c->q_tail = c->n_rec = c->n_def = c->conv_tail = 0;
  }
  const int prev_dir = c->fresh ? 0 : c->dir;
  c->fresh = 0;
  // a BFS has fewer than n levels: a frontier still non-empty past level n
  // can only come from a fault in the step kernels, and ends the loop with
  // an error instead of running on
  if (c->n_f != 0 && (int64_t)c->level > A.n) c->overflow = 2;
  if (c->n_f == 0 || c->overflow == 2) {
    c->done = 1;
    c->n_levels = c->level;
    return kCaseNone;
  }
  int dir = 0;
  switch (c->mode) {
    case DOBFS_DIR_TOPDOWN: dir = 0; break;
    case DOBFS_DIR_BOTTOMUP: dir = 1; break;
    case DOBFS_DIR_RANDOM: dir = (int)(gen_mix64(c->sched_seed ^ (uint64_t)c->level) & 1ull); break;
    case DOBFS_DIR_STATIC:
      if (prev_dir == 0) {
        // next frontier estimated as static_pct percent of the frontier's out-edges
        const int64_t est = c->m_f * (int64_t)c->static_pct / 100;
        dir = (est * (int64_t)c->beta > A.n) ? 1 : 0;
      } else {
        dir = (c->bu_run >= c->bu_steps) ? 0 : 1;
      }
      break;
    default:  // alpha/beta
      if (prev_dir == 0)
        dir = (c->m_f * (int64_t)c->alpha > c->m_u) ? 1 : 0;
      else
        dir = (c->n_f * (int64_t)c->beta < A.n && c->n_f < c->n_f_prev) ? 0 : 1;
      break;
  }
  int kase;
  c->split_w = 0;
  if (dir == 0) {
    // heavy top-down levels mark a bitmap and recover parents afterwards
    const bool bm = c->td_bm_div > 0 && c->m_f * (int64_t)c->td_bm_div >= A.n;
    kase = bm ? (c->fmt == 0 ? 4 : 5) : (c->fmt == 0 ? 0 : 2);
    if (bm && A.o2n && c->td_split_pct > 0 && c->m_f > 0) {
      // mixed level: a vertex of degree d receives about d * m_f / nnz of the
      // frontier's edges, so top-down pays that many probes for it, a bottom-up
      // search about one (its first neighbours are the hubs). Vertices of degree
      // >= 2^k >= td_split_pct/100 * nnz / m_f (a prefix of the degree-sorted
      // IDs) are searched bottom-up; the rows' entries beyond them go top-down.
      const double dx = (double)c->td_split_pct * (double)A.nnz / (100.0 * (double)c->m_f);
      int k = 0;
      while (k < 32 && (double)(1ll << k) < dx) ++k;
      c->split_w = (A.deg_ge[k] >> 10) << 5;  // whole groups of 32 words
    }
  } else {
    kase = (c->fmt == 1) ? 1 : 3;
  }
  c->dir = dir;
  c->step_case = kase;
  return kase;
}

// The switch of the fused loop works on a copy of the control block read
// from L2 in one batch of loads (the other SMs' atomics reach the block
// through L2 while this SM runs on) and writes it back whole; nothing else
// touches the block while the switch runs.
template <class OffT>
__device__ int switch_body_coherent(const BfsArgs<OffT>& A) {
  static_assert(sizeof(BfsCtl) % 4 == 0, "control block in words");
  BfsCtl lc;
#pragma unroll
  for (int i = 0; i < (int)(sizeof(BfsCtl) / 4); ++i)
    reinterpret_cast<uint32_t*>(&lc)[i] = __ldcg(reinterpret_cast<const uint32_t*>(A.ctl) + i);
  const int kase = switch_decide(A, &lc);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(BfsCtl) / 4); ++i)
    reinterpret_cast<uint32_t*>(A.ctl)[i] = reinterpret_cast<const uint32_t*>(&lc)[i];
  return kase;
}

template <class OffT>
__global__ void k_switch(BfsArgs<OffT> A, cudaGraphConditionalHandle h_while, cudaGraphConditionalHandle h_case,
                         int in_graph) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int kase = switch_decide(A, A.ctl);
  if (in_graph) {
    cudaGraphSetConditional(h_case, (unsigned)kase);
    if (kase == kCaseNone) cudaGraphSetConditional(h_while, 0);
  }
}

// Top-down, part 1: short rows expanded in place, long rows cut into
// chunk records.
template <class OffT, bool BM, int NT, bool COH>
__device__ __forceinline__ void td_bin_body(const BfsArgs<OffT>& A, const BfsCtl* c) {
  __shared__ unsigned long long sh[NT / 32];
  const int32_t L = c->level;
  const int64_t nf = c->n_f;
  const int32_t* cur = (L & 1) ? A.q1 : A.q0;
  int32_t* nxt = (L & 1) ? A.q0 : A.q1;
  const int64_t small = c->td_small, chunk = c->td_chunk;
  // mixed level: targets below x are searched bottom-up; only the rest of
  // each (sorted) row is expanded here
  const int32_t x = BM ? (int32_t)(c->split_w << 5) : 0;
  unsigned long long m_new = 0, ex = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = bc_vid(ld_mut<COH>(cur + i), A.n, &A.ctl->bc_site, kBcTdFrontier);
    int64_t s = (int64_t)A.off[u];
    int64_t e = (int64_t)A.off[u + 1];
    bc_row(s, e, A.nnz, &A.ctl->bc_site, kBcTdRow);
    if (BM && x > 0 && e - s > small) s = lower_bound_col(A.cols, s, e, x);
    ex += (unsigned long long)(e - s);
    if (e - s <= small) {
      constexpr int kE = 4;  // entries per step (short rows: wider steps measured no faster)
      for (int64_t j = s; j < e; j += kE) {
        int32_t v[kE];
        unsigned valid = 0;
#pragma unroll
        for (int t = 0; t < kE; ++t) {
          v[t] = (j + t < e) ? bc_vid(A.cols[j + t], A.n, &A.ctl->bc_site, kBcTdColumn) : 0;
          if (j + t < e && v[t] >= x) valid |= 1u << t;
        }
        if constexpr (BM) {
          td_mark4<COH>(A, v, valid, (L & 1) ? A.fbm0 : A.fbm1);
        } else {
          unsigned won = td_claimN<kE>(A, v, valid, u, L + 1, m_new);
          while (won) {
            const int t = __ffs(won) - 1;
            won &= won - 1;
            enqueue(&A.ctl->q_tail, nxt, v[t], A.n, &A.ctl->bc_site, kBcTdQueue);
          }
        }
      }
    } else {
      const int64_t a = s & ~3ll;
      const unsigned nch = (unsigned)ceil_div(e - a, chunk);
      const unsigned base = atomicAdd(&A.ctl->n_rec, nch);
      if ((int64_t)base + nch > A.rec_cap) {
        A.ctl->overflow = 1;
        continue;
      }
      if (BM) {
        // marking needs no parent: the record holds the chunk's position
        // (start, length, entries to skip before the row's part starts)
        unsigned long long* r64 = reinterpret_cast<unsigned long long*>(A.rec);
        for (unsigned k = 0; k < nch; ++k) {
          const int64_t lo = a + (int64_t)k * chunk;
          const int64_t hi = min(e, lo + chunk);
          r64[base + k] = ((unsigned long long)lo << 16) | ((unsigned long long)(hi - lo) << 2) |
                          (unsigned long long)(max(s, lo) - lo);
        }
      } else {
        for (unsigned k = 0; k < nch; ++k) A.rec[base + k] = make_int2(u, (int)k);
      }
    }
  }
  m_new = block_sum_u64(m_new, sh);
  ex = block_sum_u64(ex, sh);
  if (threadIdx.x == 0) {
    if (m_new) atomicAdd(&A.ctl->nx_m, m_new);
    if (ex) atomicAdd(&A.ctl->nx_examined, ex);
  }
}

template <class OffT, bool BM, int NT>
__global__ void __launch_bounds__(NT) k_td_bin(BfsArgs<OffT> A) {
  td_bin_body<OffT, BM, NT, false>(A, A.ctl);
}

// Top-down, part 2: one warp per chunk record, 16-byte column loads.
template <class OffT, bool BM, int NT, bool COH>
__device__ __forceinline__ void td_chunks_body(const BfsArgs<OffT>& A, const BfsCtl* c) {
  __shared__ unsigned long long sh[NT / 32];
  const int32_t L = c->level;
  const int64_t nrec = min((int64_t)c->n_rec, A.rec_cap);
  const int64_t chunk = c->td_chunk;
  int32_t* nxt = (L & 1) ? A.q0 : A.q1;
  unsigned long long m_new = 0;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const unsigned lane = lane_id();
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < nrec; r += warps) {
    int32_t u = 0;
    int64_t lo, hi, lo_ok;
    if (BM) {
      const unsigned long long rc = ld_mut<COH>(reinterpret_cast<const unsigned long long*>(A.rec) + r);
      lo = (int64_t)(rc >> 16);
      hi = lo + (int64_t)((rc >> 2) & 0x3FFFu);
      bc_row(lo, hi, A.nnz, &A.ctl->bc_site, kBcTdRecord);
      lo_ok = lo + (int64_t)(rc & 3u);
    } else {
      const int2 rc = ld_mut<COH>(A.rec + r);
      u = bc_vid(rc.x, A.n, &A.ctl->bc_site, kBcTdRecord);
      int64_t s = (int64_t)A.off[u], e = (int64_t)A.off[u + 1];
      bc_row(s, e, A.nnz, &A.ctl->bc_site, kBcTdRow);
      lo = (s & ~3ll) + (int64_t)rc.y * chunk;
      hi = min(e, lo + chunk);
      lo_ok = max(s, lo);
    }
    constexpr int kE = BM ? 4 : kTdClaimPer;  // entries per lane per step
    for (int64_t pb = lo; pb < hi; pb += 32 * kE) {  // uniform trip count: the warp enqueues together
      const int64_t p = pb + kE * (int64_t)lane;
      int32_t v[kE];
      unsigned valid = 0;
#pragma unroll
      for (int h = 0; h < kE; h += 4) {
        int4 x = make_int4(0, 0, 0, 0);
        if (p + h < hi) x = *reinterpret_cast<const int4*>(A.cols + p + h);
        v[h] = bc_vid(x.x, A.n, &A.ctl->bc_site, kBcTdColumn);
        v[h + 1] = bc_vid(x.y, A.n, &A.ctl->bc_site, kBcTdColumn);
        v[h + 2] = bc_vid(x.z, A.n, &A.ctl->bc_site, kBcTdColumn);
        v[h + 3] = bc_vid(x.w, A.n, &A.ctl->bc_site, kBcTdColumn);
      }
#pragma unroll
      for (int t = 0; t < kE; ++t)
        if (p + t >= lo_ok && p + t < hi) valid |= 1u << t;
      if constexpr (BM) {
        if (valid) td_mark4<COH>(A, v, valid, (L & 1) ? A.fbm0 : A.fbm1);
        continue;
      }
      const unsigned won = valid ? td_claimN<kE>(A, v, valid, u, L + 1, m_new) : 0u;
      const unsigned cnt = (unsigned)__popc(won);
      unsigned incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
      if (total) {
        unsigned qb = 0;
        if (lane == 31) qb = atomicAdd(&A.ctl->q_tail, total);
        qb = __shfl_sync(0xffffffffu, qb, 31);
        unsigned pos = qb + incl - cnt;
#pragma unroll
        for (int t = 0; t < kE; ++t)
          if ((won >> t) & 1u) {
            if (bc_pos(pos, A.n, &A.ctl->bc_site, kBcTdQueue)) nxt[pos] = v[t];
            ++pos;
          }
      }
    }
  }
  m_new = block_sum_u64(m_new, sh);
  if (threadIdx.x == 0 && m_new) atomicAdd(&A.ctl->nx_m, m_new);
}

template <class OffT, bool BM, int NT>
__global__ void __launch_bounds__(NT) k_td_chunks(BfsArgs<OffT> A) {
  td_chunks_body<OffT, BM, NT, false>(A, A.ctl);
}

// Frontier bitmap of level L -> queue of level L (after a bottom-up level,
// before a top-down one). A warp converts 32 consecutive words.
template <class OffT, bool COH>
__device__ __forceinline__ void bitmap_to_queue_body(const BfsArgs<OffT>& A, const BfsCtl* c) {
  const int32_t L = c->level;
  const uint32_t* bm = (L & 1) ? A.fbm1 : A.fbm0;
  int32_t* q = (L & 1) ? A.q1 : A.q0;
  const unsigned lane = lane_id();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; w0 < A.cand_words; w0 += stride) {
    const int64_t w = w0 + lane;
    uint32_t x = (w < A.cand_words) ? ld_mut<COH>(bm + w) : 0u;
    const unsigned cnt = (unsigned)__popc(x);
    unsigned inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
      if ((int)lane >= o) inc += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, inc, 31);
    unsigned base = 0;
    if (lane == 31 && total) base = atomicAdd(&A.ctl->conv_tail, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    unsigned pos = base + inc - cnt;
    while (x) {
      const int b = __ffs(x) - 1;
      x &= x - 1;
      if (bc_pos(pos, A.n, &A.ctl->bc_site, kBcConvert)) q[pos] = (int32_t)(w * 32 + b);
      ++pos;
    }
  }
}

template <class OffT>
__global__ void __launch_bounds__(kThreads) k_bitmap_to_queue(BfsArgs<OffT> A) {
  bitmap_to_queue_body<OffT, false>(A, A.ctl);
}

// Queue of level L -> frontier bitmap of level L (after a top-down level,
// before a bottom-up one). Both bitmaps were cleared just before.
template <class OffT, bool COH>
__device__ __forceinline__ void queue_to_bitmap_body(const BfsArgs<OffT>& A, const BfsCtl* c) {
  const int32_t L = c->level;
  const int64_t nf = c->n_f;
  uint32_t* bm = (L & 1) ? A.fbm1 : A.fbm0;
  const int32_t* q = (L & 1) ? A.q1 : A.q0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = bc_vid(ld_mut<COH>(q + i), A.n, &A.ctl->bc_site, kBcConvert);
    atomicOr(bm + (v >> 5), 1u << (v & 31));
  }
}

template <class OffT>
__global__ void __launch_bounds__(kThreads) k_queue_to_bitmap(BfsArgs<OffT> A) {
  queue_to_bitmap_body<OffT, false>(A, A.ctl);
}

// Bottom-up, part 1 (Algorithm 1, bottom-up branch). A warp takes 32
// consecutive visited words (1024 vertices) at a time: one coalesced load of
// the visited and isolated words gives the candidates (unvisited vertices
// with an edge), which are compacted so that every lane holds one candidate
// per round. First pass: every candidate tests its first neighbour, read
// with its degree from the packed (first, degree) array; rows are sorted
// with the highest-degree neighbour first, so most vertices that have a
// frontier neighbour resolve with that one 8-byte load. Second pass, over
// the misses only (so a long scan does not hold up the first tests of the
// other candidates): each scans the rest of its first bu_scan entries, four
// loads at a time, and stops at the first neighbour in the frontier; longer
// rows without a hit go to the deferred list. Found vertices are collected
// per word in shared memory and every lane writes its own next-frontier and
// visited word: no global atomics.
template <class OffT, bool RECOVER, int NT, bool COH>
__device__ __forceinline__ void bu_body(const BfsArgs<OffT>& A, const BfsCtl* c) {
  __shared__ unsigned long long sh[NT / 32];
  __shared__ uint32_t s_found[NT / 32][32];
  __shared__ uint16_t s_cand[NT / 32][1024];
  __shared__ int64_t s_tab[2 * kSmallDeg];
  if (threadIdx.x < 2 * kSmallDeg) s_tab[threadIdx.x] = A.small_deg ? A.small_tab[threadIdx.x] : 0;
  __syncthreads();
  const int32_t L = c->level;
  const uint32_t* front = (L & 1) ? A.fbm1 : A.fbm0;
  uint32_t* next = (L & 1) ? A.fbm0 : A.fbm1;
  const int32_t scan = c->bu_scan;
  const unsigned lane = lane_id();
  const int wid = threadIdx.x >> 5;
  unsigned long long n_new = 0, m_new = 0, ex = 0, sc = 0;
  // words searched: all candidates in a bottom-up level; in a bitmap-output
  // top-down level, the search covers [0, split_w) (the mixed level's
  // bottom-up part; empty otherwise) and the parent recovery the rest
  const int64_t split = c->split_w;
  const int64_t w_lo = RECOVER ? split : 0;
  const int64_t w_hi = RECOVER ? A.cand_words : (c->step_case >= 4 ? split : A.cand_words);
  const int64_t groups = ceil_div(w_hi, 32);
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t grp = w_lo / 32 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); grp < groups;
       grp += warps) {
    const int64_t w = grp * 32 + lane;
    const bool in = w < w_hi;
    const uint32_t vis = in ? ld_mut<COH>(A.visited + w) : ~0u;
    // recovery: the candidates are the vertices the top-down marking found
    const uint32_t cand = in ? (RECOVER ? ld_mut<COH>(next + w) : ~(vis | A.iso[w])) : 0u;
    const unsigned cnt = (unsigned)__popc(cand);
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)lane >= o) incl += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    s_found[wid][lane] = 0u;
    __syncwarp();
    sc += cnt;
    // candidate list: each lane writes the positions (word << 5 | bit) of its
    // word's candidates at its exclusive prefix
    {
      uint32_t x = cand;
      unsigned pos = incl - cnt;
      while (x) {
        const unsigned b = (unsigned)(__ffs(x) - 1);
        x &= x - 1;
        s_cand[wid][pos++] = (uint16_t)((lane << 5) | b);
      }
    }
    __syncwarp();
    // phase 1: every candidate tests its first neighbour (two per lane per
    // round); the misses are compacted at the front of the candidate list
    unsigned n_miss = 0;
    for (unsigned base = 0; base < total; base += 64) {
      unsigned loc[2];
      int32_t vv[2];
      bool act[2];
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2) {
        const unsigned k = base + 32 * c2 + lane;
        act[c2] = k < total;
        loc[c2] = act[c2] ? (unsigned)s_cand[wid][k] : 0u;
        vv[c2] = (int32_t)(grp * 1024 + loc[c2]);
      }
      int2 fd[2];
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2) {
        fd[c2] = act[c2] ? __ldg(A.firstdeg + vv[c2]) : make_int2(0, 0);
        if (act[c2]) fd[c2].x = bc_vid(fd[c2].x, A.n, &A.ctl->bc_site, kBcBuFirst);
      }
      bool hit0[2];
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2) hit0[c2] = act[c2] && test_bit<COH>(front, fd[c2].x);
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2) {
        if (act[c2]) ex += 1;
        if (hit0[c2]) {
          atomicOr(&s_found[wid][loc[c2] >> 5], 1u << (loc[c2] & 31u));
          A.lp[vv[c2]] = make_int2(L + 1, fd[c2].x);
          n_new += 1;
          m_new += (unsigned long long)fd[c2].y;
        }
        // the list slots written here were read in this or an earlier round
        const bool miss = act[c2] && !hit0[c2] && fd[c2].y > 1;
        const unsigned bal = __ballot_sync(0xffffffffu, miss);
        if (miss) s_cand[wid][n_miss + __popc(bal & lanemask_lt())] = (uint16_t)loc[c2];
        n_miss += (unsigned)__popc(bal);
      }
    }
    __syncwarp();
    // phase 2: the misses scan the rest of their first bu_scan entries, four
    // loads at a time, and stop at the first neighbour in the frontier;
    // longer rows without a hit go to the deferred list
    for (unsigned base = 0; base < n_miss; base += 32) {
      const unsigned k = base + lane;
      if (k >= n_miss) continue;
      const unsigned lc = (unsigned)s_cand[wid][k];
      const int32_t v = (int32_t)(grp * 1024 + lc);
      const int32_t dv = __ldg(&A.firstdeg[v].y);
      // small degrees: the row start follows from the ID (no offset load)
      int64_t s0 = dv < A.small_deg ? s_tab[dv] + (int64_t)(v - (int32_t)s_tab[kSmallDeg + dv]) * dv
                                    : (int64_t)A.off[v];
      int64_t e0 = s0 + dv;
      bc_row(s0, e0, A.nnz, &A.ctl->bc_site, kBcBuRow);
      const int64_t lim = s0 + min(e0 - s0, (int64_t)scan);
      int32_t parent = -1;
      for (int64_t p = s0 + 1; p < lim && parent < 0; p += 4) {
        int32_t u[4];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          u[t] = (p + t < lim) ? bc_vid(A.cols[p + t], A.n, &A.ctl->bc_site, kBcBuColumn) : -1;
        bool h[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) h[t] = (u[t] >= 0) && test_bit<COH>(front, u[t]);
#pragma unroll
        for (int t = 3; t >= 0; --t)
          if (h[t]) parent = u[t];
        ex += (unsigned long long)min((int64_t)4, lim - p);
      }
      if (parent >= 0) {
        atomicOr(&s_found[wid][lc >> 5], 1u << (lc & 31u));
        A.lp[v] = make_int2(L + 1, parent);
        n_new += 1;
        m_new += (unsigned long long)dv;
      } else if (dv > scan) {
        enqueue(&A.ctl->n_def, A.def, v, A.n, &A.ctl->bc_site, kBcBuDeferred);
      }
    }
    __syncwarp();
    if (in) {
      const uint32_t f = s_found[wid][lane];
      if (!RECOVER) next[w] = f;
      if (f) A.visited[w] = vis | f;
    }
    __syncwarp();
  }
  n_new = block_sum_u64(n_new, sh);
  m_new = block_sum_u64(m_new, sh);
  ex = block_sum_u64(ex, sh);
  sc = block_sum_u64(sc, sh);
  if (threadIdx.x == 0) {
    if (n_new) atomicAdd(&A.ctl->nx_n, n_new);
    if (m_new) atomicAdd(&A.ctl->nx_m, m_new);
    if (ex) atomicAdd(&A.ctl->nx_examined, ex);
    if (sc) atomicAdd(&A.ctl->nx_scanned, sc);
  }
}

template <class OffT, bool RECOVER, int NT>
__global__ void __launch_bounds__(NT, bu_min_blocks(NT)) k_bu(BfsArgs<OffT> A) {
  bu_body<OffT, RECOVER, NT, false>(A, A.ctl);
}

// Clears the next-frontier bitmap of level L (bitmap-output top-down step
// after a bottom-up level, when the current frontier bitmap must stay).
template <class OffT>
__device__ __forceinline__ void clear_next_body(const BfsArgs<OffT>& A, const BfsCtl* c) {
  const int32_t L = c->level;
  uint32_t* next = (L & 1) ? A.fbm0 : A.fbm1;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < A.words; w += (int64_t)gridDim.x * blockDim.x)
    next[w] = 0u;
}

template <class OffT>
__global__ void k_clear_next(BfsArgs<OffT> A) {
  clear_next_body(A, A.ctl);
}

// Bottom-up, part 2: rows with no frontier neighbour among their first bu_scan
// entries; one warp per row, 16-byte loads, the ballot picks the first hit
// in row order.
template <class OffT, bool COH>
__device__ __forceinline__ void bu_long_body(const BfsArgs<OffT>& A, const BfsCtl* c) {
  __shared__ unsigned long long sh[kThreads / 32];
  const int32_t L = c->level;
  const int64_t nd = c->n_def;
  const uint32_t* front = (L & 1) ? A.fbm1 : A.fbm0;
  uint32_t* next = (L & 1) ? A.fbm0 : A.fbm1;
  const unsigned lane = lane_id();
  unsigned long long n_new = 0, m_new = 0, ex = 0;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < nd; i += warps) {
    const int32_t v = bc_vid(ld_mut<COH>(A.def + i), A.n, &A.ctl->bc_site, kBcBuDeferred);
    int64_t s0 = (int64_t)A.off[v], e = (int64_t)A.off[v + 1];
    bc_row(s0, e, A.nnz, &A.ctl->bc_site, kBcBuRow);
    const int64_t s = s0 + c->bu_scan;
    int32_t parent = -1;
    for (int64_t base = s & ~3ll; base < e; base += 128) {
      const int64_t p = base + 4 * (int64_t)lane;
      int32_t hit = -1;
      if (p < e) {
        const int4 x = *reinterpret_cast<const int4*>(A.cols + p);
        const int32_t us[4] = {bc_vid(x.x, A.n, &A.ctl->bc_site, kBcBuColumn),
                               bc_vid(x.y, A.n, &A.ctl->bc_site, kBcBuColumn),
                               bc_vid(x.z, A.n, &A.ctl->bc_site, kBcBuColumn),
                               bc_vid(x.w, A.n, &A.ctl->bc_site, kBcBuColumn)};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int64_t idx = p + t;
          if (hit < 0 && idx >= s && idx < e && test_bit<COH>(front, us[t])) hit = us[t];
        }
      }
      const unsigned b = __ballot_sync(0xffffffffu, hit >= 0);
      { const int64_t span = min(e, base + 128) - max(s, base); ex += (unsigned long long)(span > 0 ? span : 0); }
      if (b) {
        parent = __shfl_sync(0xffffffffu, hit, __ffs(b) - 1);
        break;
      }
    }
    if (parent >= 0 && lane == 0) {
      atomicOr(next + (v >> 5), 1u << (v & 31));
      atomicOr(A.visited + (v >> 5), 1u << (v & 31));
      A.lp[v] = make_int2(L + 1, parent);
      n_new += 1;
      m_new += (unsigned long long)(e - s0);
    }
  }
  if (lane != 0) ex = 0;
  n_new = block_sum_u64(n_new, sh);
  m_new = block_sum_u64(m_new, sh);
  ex = block_sum_u64(ex, sh);
  if (threadIdx.x == 0) {
    if (n_new) atomicAdd(&A.ctl->nx_n, n_new);
    if (m_new) atomicAdd(&A.ctl->nx_m, m_new);
    if (ex) atomicAdd(&A.ctl->nx_examined, ex);
  }
}

template <class OffT>
__global__ void __launch_bounds__(kThreads) k_bu_long(BfsArgs<OffT> A) {
  bu_long_body<OffT, false>(A, A.ctl);
}

// Results in original IDs: level_out[o], parent_out[o] for every vertex.
// Each thread handles four consecutive original IDs (16-byte map loads and
// output stores). Vertices renumbered past the last one with an edge are
// isolated: unreached unless they are the root, so only the root among them
// needs the visited bit and the (level, parent) gather.
template <class OffT, int NT>
__global__ void __launch_bounds__(NT) k_output(BfsArgs<OffT> A, const int32_t* __restrict__ n2o,
                                                     int32_t root_orig, int32_t* __restrict__ level_out,
                                                     int32_t* __restrict__ parent_out) {
  constexpr int kQ = 2;  // quads per thread and step: eight independent gathers in flight
  constexpr int64_t kOutChunk = 2048;  // quads per chunk (8192 original IDs)
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // the fused level loop (done by now): report a barrier that timed out
    // and reset the barrier for the next run
    if (A.gbar[2]) A.ctl->overflow = 3;
    A.gbar[0] = 0u;
    A.gbar[2] = 0u;
  }
  const int32_t root = A.o2n ? __ldg(A.o2n + root_orig) : root_orig;
  const int64_t quads = A.n >> 2;
  const bool vec = ((reinterpret_cast<uintptr_t>(level_out) | reinterpret_cast<uintptr_t>(parent_out)) & 15) == 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // blocks take chunks of kOutChunk quads in turn (one counter): each block
  // streams a contiguous stretch of the map and the outputs
  __shared__ int64_t s_chunk;
  for (;;) {
    if (threadIdx.x == 0) s_chunk = (int64_t)atomicAdd(&A.ctl->out_next, 1u);
    __syncthreads();
    const int64_t qlo = s_chunk * kOutChunk, qhi = min(quads, qlo + kOutChunk);
    __syncthreads();
    if (qlo >= quads) break;
    for (int64_t q0 = qlo + threadIdx.x; q0 < qhi; q0 += (int64_t)blockDim.x * kQ) {
      int32_t v[kQ][4];
      bool inq[kQ];
#pragma unroll
      for (int a = 0; a < kQ; ++a) {
        const int64_t q = q0 + a * (int64_t)blockDim.x;
        inq[a] = q < qhi;
        if (A.o2n) {
          const int4 m = inq[a] ? __ldg(reinterpret_cast<const int4*>(A.o2n) + q) : make_int4(0, 0, 0, 0);
          v[a][0] = bc_vid(m.x, A.n, &A.ctl->bc_site, kBcOutput);
          v[a][1] = bc_vid(m.y, A.n, &A.ctl->bc_site, kBcOutput);
          v[a][2] = bc_vid(m.z, A.n, &A.ctl->bc_site, kBcOutput);
          v[a][3] = bc_vid(m.w, A.n, &A.ctl->bc_site, kBcOutput);
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t) v[a][t] = (int32_t)(q * 4 + t);
        }
      }
      // a vertex renumbered past the last one with an edge is isolated: only
      // the root among them can be reached
      bool need[kQ][4];
      uint32_t vw[kQ][4];
      int2 x[kQ][4];
#pragma unroll
      for (int a = 0; a < kQ; ++a)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int32_t vt = v[a][t];
          need[a][t] = inq[a] && (!A.o2n || vt < A.n_nonisolated || vt == root);
          // the visited word and the (level, parent) pair are loaded together;
          // the pair is used only if the vertex was visited
          vw[a][t] = need[a][t] ? __ldg(A.visited + (vt >> 5)) : 0u;
          x[a][t] = need[a][t] ? A.lp[vt] : make_int2(-1, -1);
        }
      int32_t lev[kQ][4], par[kQ][4];
#pragma unroll
      for (int a = 0; a < kQ; ++a)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const bool vis = (vw[a][t] >> (v[a][t] & 31)) & 1u;
          lev[a][t] = vis ? x[a][t].x : -1;
          const int32_t py = vis ? bc_vid(x[a][t].y, A.n, &A.ctl->bc_site, kBcOutput) : 0;
          par[a][t] = vis ? (n2o ? __ldg(n2o + py) : py) : -1;
        }
#pragma unroll
      for (int a = 0; a < kQ; ++a) {
        if (!inq[a]) continue;
        const int64_t q = q0 + a * (int64_t)blockDim.x;
        if (vec) {
          reinterpret_cast<int4*>(level_out)[q] = make_int4(lev[a][0], lev[a][1], lev[a][2], lev[a][3]);
          if (parent_out)
            reinterpret_cast<int4*>(parent_out)[q] = make_int4(par[a][0], par[a][1], par[a][2], par[a][3]);
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            level_out[q * 4 + t] = lev[a][t];
            if (parent_out) parent_out[q * 4 + t] = par[a][t];
          }
        }
      }
    }
  }
  for (int64_t o = quads * 4 + tid; o < A.n; o += stride) {  // ragged tail
    const int32_t vt = A.o2n ? bc_vid(__ldg(A.o2n + o), A.n, &A.ctl->bc_site, kBcOutput) : (int32_t)o;
    int32_t lev = -1, par = -1;
    if ((__ldg(A.visited + (vt >> 5)) >> (vt & 31)) & 1u) {
      const int2 y = A.lp[vt];
      lev = y.x;
      const int32_t py = bc_vid(y.y, A.n, &A.ctl->bc_site, kBcOutput);
      par = n2o ? __ldg(n2o + py) : py;
    }
    level_out[o] = lev;
    if (parent_out) parent_out[o] = par;
  }
}

// Canonical parent: smallest original-ID neighbour one level up. One warp
// per vertex, over the full row.
template <class OffT>
__global__ void __launch_bounds__(kThreads) k_canonical_parent(BfsArgs<OffT> A, const int32_t* __restrict__ n2o,
                                                               int32_t* __restrict__ parent_out) {
  const unsigned lane = lane_id();
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < A.n; v += warps) {
    if (!((__ldg(A.visited + (v >> 5)) >> (v & 31)) & 1u)) continue;
    const int32_t lev = A.lp[v].x;
    if (lev <= 0) continue;
    int64_t s = (int64_t)A.off[v], e = (int64_t)A.off[v + 1];
    bc_row(s, e, A.nnz, &A.ctl->bc_site, kBcOutput);
    int32_t best = INT32_MAX;
    for (int64_t j = s + lane; j < e; j += 32) {
      const int32_t u = bc_vid(A.cols[j], A.n, &A.ctl->bc_site, kBcOutput);
      if (((__ldg(A.visited + (u >> 5)) >> (u & 31)) & 1u) && A.lp[u].x == lev - 1) {
        const int32_t o = n2o ? n2o[u] : u;
        best = min(best, o);
      }
    }
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xffffffffu, best, o));
    if (lane == 0) parent_out[n2o ? n2o[v] : v] = best;
  }
}

// (first neighbour, degree) of every vertex, for the bottom-up first test.
template <class OffT>
__global__ void k_firstdeg(const OffT* __restrict__ off, const int32_t* __restrict__ cols, int64_t n,
                           int2* __restrict__ fd) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = (int64_t)off[v], e = (int64_t)off[v + 1];
    fd[v] = make_int2(e > s ? cols[s] : -1, (int32_t)(e - s));
  }
}

// ------------------------------------------------------------------ fused loop
// The level loop of a small graph in one cooperative kernel: per level the
// step kind's phases, separated by grid-wide barriers instead of kernel
// launches (a level of a small graph costs its launches more than its
// work); the last block to reach a level's final barrier runs the switch
// (one thread) before the others leave it. Every block takes the same path:
// the step kind and the end of the loop are read from the control block
// after a barrier, from L2, into shared memory (s_c), and the phases read
// the control fields from that copy; data the loop writes is read from L2
// too (the bodies' COH loads). The loop ends at the switch's end mark, or
// after n + 2 levels at most (a fault; the switch flags it past n).
//
// The cooperative launch makes every block resident at once, so each
// barrier completes once all blocks reach it; a block still waits at most
// kGridBarrierNs there. A wait that runs out (never expected) sets the
// timed-out flag and ends that block's loop; the others then run out at
// their next barrier. The output kernel that follows every run reports the
// flag in the control block and resets the barrier.
constexpr int64_t kFusedMaxNonisolated = int64_t(1) << 21;  // graphs this size or smaller use the fused loop
constexpr int64_t kFusedMaxNnz = int64_t(1) << 27;          // ... with at most this many stored entries
constexpr unsigned long long kGridBarrierNs = 2000000000ull;  // longest wait at a barrier (2 s)
constexpr size_t kGridBarBytes = 16;                          // after the control block

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of `nblocks` blocks (all resident): bar[0] counts the
// blocks that arrived, bar[1] is the generation the last of them advances,
// bar[2] the timed-out flag. `gen` (thread 0's copy of the generation)
// advances with every barrier. The last block to arrive runs `last` (one
// thread) before it lets the others go: every block's writes before the
// barrier are visible to it then. Returns false in every thread of the
// block if the wait ran out (kGridBarrierNs).
template <class Last>
__device__ __forceinline__ bool grid_barrier(uint32_t* bar, uint32_t& gen, uint32_t nblocks, Last&& last) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    uint32_t old;
    // arrival: releases the block's writes (ordered before it by the block
    // barrier) and, in the last block, acquires every other block's
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
    if (old == nblocks - 1) {
      last();
      atomicExch(bar, 0u);  // the count starts over for the next barrier
      // releases the hook's writes and the reset with the new generation
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(bar + 1), "r"(gen + 1u) : "memory");
    } else {
      const unsigned long long t0 = globaltimer_ns();
      for (uint32_t k = 1; ld_acquire_gpu(bar + 1) == gen; ++k) {
        if ((k & 255u) == 0 && globaltimer_ns() - t0 > kGridBarrierNs) {
          atomicExch(bar + 2, 1u);
          ok = 0;
          break;
        }
      }
    }
    gen += 1u;  // the waiting blocks' acquire loads order their later reads
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The fused loop's hooks: status init and/or the direction switch.
enum { kHookNone = 0, kHookSwitch = 1, kHookInitSwitch = 2 };

template <class OffT>
__device__ __forceinline__ bool fused_barrier(const BfsArgs<OffT>& A, uint32_t& gen, int hook, const RunParams* P) {
  return grid_barrier(A.gbar, gen, gridDim.x, [&] {
    if (hook == kHookInitSwitch) {
      init_body(A, *P);
      __threadfence();
    }
    if (hook != kHookNone) switch_body_coherent(A);
  });
}

// Self-test of the barrier: `rounds` barriers over the launched blocks, or
// over one block more than launched (`missing`), so that every wait runs
// out. Before each barrier every block adds one to cnt[0]; after it block 0
// checks that all blocks did (cnt[1] counts the rounds that passed, cnt[2]
// the rounds that saw a short count).
__global__ void __launch_bounds__(kThreads) k_barrier_probe(uint32_t* bar, uint32_t* cnt, uint32_t rounds,
                                                          uint32_t missing) {
  uint32_t gen = threadIdx.x == 0 ? ld_acquire_gpu(bar + 1) : 0u;
  const uint32_t nb = gridDim.x + missing;
  for (uint32_t r = 0; r < rounds; ++r) {
    if (threadIdx.x == 0) atomicAdd(cnt, 1u);
    if (!grid_barrier(bar, gen, nb, [] {})) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (__ldcg(cnt) != gridDim.x * (r + 1)) atomicAdd(cnt + 2, 1u);
      atomicAdd(cnt + 1, 1u);
    }
    // no block adds for the next round before block 0 has checked this one
    if (!grid_barrier(bar, gen, nb, [] {})) return;
  }
}

template <class OffT>
__device__ __forceinline__ void load_ctl(BfsCtl* dst, const BfsCtl* src) {
  static_assert(sizeof(BfsCtl) % 4 == 0, "control block in words");
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  const uint32_t* g = reinterpret_cast<const uint32_t*>(src);
  for (int i = threadIdx.x; i < (int)(sizeof(BfsCtl) / 4); i += blockDim.x) d[i] = __ldcg(g + i);
  __syncthreads();
}

// One barrier between levels: its last block closes the level and picks the
// next step (the switch) before the others leave it.
template <class OffT>
// one block per SM: the registers a thread may use are not capped for occupancy
__global__ void __launch_bounds__(kThreads, 1) k_bfs_fused(BfsArgs<OffT> A, RunParams P) {
  __shared__ BfsCtl s_c;
  // thread 0's generation: read before this block's first arrival, which
  // no barrier completes without
  uint32_t gen = threadIdx.x == 0 ? ld_acquire_gpu(A.gbar + 1) : 0u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
#define FUSED_BARRIER(hook) \
  if (!fused_barrier(A, gen, hook, &P)) return
  for (int64_t w = tid; w < A.words; w += stride) A.visited[w] = 0u;
  FUSED_BARRIER(kHookInitSwitch);
  for (int64_t it = 0; it <= A.n + 1; ++it) {
    load_ctl<OffT>(&s_c, A.ctl);
    if (s_c.done) break;
    const int kase = s_c.step_case;
    if (kase == 2 || kase == 5) {  // frontier as a bitmap, the step needs a queue
      bitmap_to_queue_body<OffT, true>(A, &s_c);
      if (kase == 5) clear_next_body(A, &s_c);
      FUSED_BARRIER(kHookNone);
      load_ctl<OffT>(&s_c, A.ctl);
    }
    if (kase == 3 || kase == 4) {  // frontier as a queue, the step needs both bitmaps cleared and the frontier's
      uint32_t* f = A.fbm0;         // fbm1 follows fbm0
      for (int64_t w = tid; w < 2 * A.words; w += stride) f[w] = 0u;
      FUSED_BARRIER(kHookNone);
      queue_to_bitmap_body<OffT, true>(A, &s_c);
      FUSED_BARRIER(kHookNone);
      load_ctl<OffT>(&s_c, A.ctl);
    }
    if (kase == 0 || kase == 2) {
      td_bin_body<OffT, false, kThreads, true>(A, &s_c);
      FUSED_BARRIER(kHookNone);
      load_ctl<OffT>(&s_c, A.ctl);
      td_chunks_body<OffT, false, kThreads, true>(A, &s_c);
    } else if (kase == 1 || kase == 3) {
      bu_body<OffT, false, kThreads, true>(A, &s_c);
      FUSED_BARRIER(kHookNone);
      load_ctl<OffT>(&s_c, A.ctl);
      bu_long_body<OffT, true>(A, &s_c);
    } else {  // 4, 5: top-down marking a bitmap, the mixed level's bottom-up part, parent recovery
      td_bin_body<OffT, true, kThreads, true>(A, &s_c);
      FUSED_BARRIER(kHookNone);
      load_ctl<OffT>(&s_c, A.ctl);
      td_chunks_body<OffT, true, kThreads, true>(A, &s_c);
      bu_body<OffT, false, kThreads, true>(A, &s_c);
      FUSED_BARRIER(kHookNone);
      load_ctl<OffT>(&s_c, A.ctl);
      bu_body<OffT, true, kThreads, true>(A, &s_c);
      FUSED_BARRIER(kHookNone);
      load_ctl<OffT>(&s_c, A.ctl);
      bu_long_body<OffT, true>(A, &s_c);
    }
    FUSED_BARRIER(kHookSwitch);
  }
#undef FUSED_BARRIER
}

int grid_cap(int per_sm) { return sm_count() * per_sm; }

// Grid of the fused loop for g: 0 if g is too large for it, else one block
// per 1,024 vertices with an edge, at most one per SM (resident at once, as
// the cooperative launch needs). A grid barrier over more blocks costs more
// than their extra warps gain: at R-MAT scale 20, 444 blocks (three per SM)
// took 0.196 ms per BFS, 148 blocks 0.182 ms.
template <class OffT>
int fused_grid_for(const dobfs_graph* g) {
  if (g->n_nonisolated > kFusedMaxNonisolated || g->nnz > kFusedMaxNnz) return 0;
  static int per_sm = -1;
  if (per_sm < 0) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bfs_fused<OffT>, kThreads, 0) != cudaSuccess) {
      cudaGetLastError();
      occ = 0;
    }
    per_sm = occ;
  }
  if (per_sm < 1) return 0;
  const int64_t want = std::max<int64_t>(1, ceil_div(std::max<int64_t>(g->n_nonisolated, 1), 1024));
  return (int)std::min<int64_t>((int64_t)sm_count(), want);
}

template <class OffT>
BfsArgs<OffT> make_args(dobfs_graph* g) {
  BfsArgs<OffT> A;
  A.off = g->off.as<OffT>();
  A.cols = g->cols.as<int32_t>();
  A.iso = g->isolated.as<uint32_t>();
  A.o2n = g->reindexed ? g->orig2new.as<int32_t>() : nullptr;
  A.firstdeg = g->firstdeg.as<int2>();
  A.deg_ge = g->degge.as<int64_t>();
  A.small_tab = g->degge.as<int64_t>() + 33;
  A.small_deg = g->small_deg;
  A.visited = g->visited.as<uint32_t>();
  A.fbm0 = g->fbm.as<uint32_t>();
  A.fbm1 = g->fbm.as<uint32_t>() + g->words;
  A.lp = g->lp.as<int2>();
  A.q0 = g->q0.as<int32_t>();
  A.q1 = g->q1.as<int32_t>();
  A.rec = g->rec.as<int2>();
  A.def = g->deferred.as<int32_t>();
  A.ctl = g->ctl.as<BfsCtl>();
  A.gbar = reinterpret_cast<uint32_t*>(g->ctl.as<char>() + sizeof(BfsCtl));
  A.trace = g->trace.as<LevelRec>();
  A.n = g->n;
  A.nnz = g->nnz;
  A.words = g->words;
  // vertices past the last one with an edge are never candidates; with
  // degree-sorted IDs these are all isolated vertices
  A.cand_words = g->reindexed ? ceil_div(std::max<int64_t>(g->n_nonisolated, 1), 32) : g->words;
  A.rec_cap = g->rec_cap;
  A.n_nonisolated = g->n_nonisolated;
  return A;
}

// Grid sizes of the level kernels (fixed: the work sizes live on the device).
struct Grids {
  int td_bin, td_chunks, conv, bu, bu_long;
};
// One full wave of resident blocks per kernel: the grid-stride loops then
// run every block to the end of the work without a second, partial wave.
template <class K>
int resident_grid(K kernel, int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 4;
  }
  fit_carveout(kernel, threads, per_sm);
  return grid_cap(per_sm);
}

// Block sizes of the step kernels: bottom-up search (bu), top-down binning
// and chunks (td).
struct BlockCfg {
  int bu = kThreads, td = kThreads;
};
BlockCfg block_cfg(const dobfs_run_opts& o) {
  BlockCfg b;
  if (o.bu_threads) b.bu = o.bu_threads;
  if (o.td_threads) b.td = o.td_threads;
  return b;
}

template <class OffT, int TB, int TT>
Grids grids() {
  static Grids G = {0, 0, 0, 0, 0};
  if (G.bu == 0) {
    G.td_bin = resident_grid(k_td_bin<OffT, false, TT>, TT);
    G.td_chunks = resident_grid(k_td_chunks<OffT, false, TT>, TT);
    G.conv = resident_grid(k_bitmap_to_queue<OffT>, kThreads);
    G.bu = resident_grid(k_bu<OffT, false, TB>, TB);
    G.bu_long = resident_grid(k_bu_long<OffT>, kThreads);
  }
  return G;
}

// The grids of graph g: a full wave of resident blocks, or fewer where g is
// too small to give every block work (the frontier, the records, the
// bitmap words and the long rows of g bound each kernel's work), so that a
// level of a small graph does not launch hundreds of idle blocks.
template <class OffT, int TB, int TT>
Grids graph_grids(const dobfs_graph* g) {
  Grids G = grids<OffT, TB, TT>();
  auto cap = [](int grid, int64_t blocks) { return (int)std::max<int64_t>(1, std::min<int64_t>(grid, blocks)); };
  const int64_t cand_words = g->reindexed ? ceil_div(std::max<int64_t>(g->n_nonisolated, 1), 32) : g->words;
  const int64_t n_front = std::max<int64_t>(g->n_nonisolated, 1);  // frontier vertices (the root counts)
  G.td_bin = cap(G.td_bin, ceil_div(n_front, TT));
  G.td_chunks = cap(G.td_chunks, ceil_div(g->rec_cap, TT / 32));
  G.conv = cap(G.conv, ceil_div(std::max(g->words, n_front), kThreads));
  G.bu = cap(G.bu, ceil_div(ceil_div(cand_words, 32), TB / 32));
  G.bu_long = cap(G.bu_long, ceil_div(std::max<int64_t>(g->deg_ge[1], 1), kThreads / 32));  // rows of >= 2 entries
  return G;
}

// Enqueues the kernels of step kind `kase` on s (used both for graph capture
// and for host-driven levels).
template <class OffT, int TB, int TT>
int launch_case_t(dobfs_graph* g, const BfsArgs<OffT>& A, int kase, cudaStream_t s, cudaEvent_t main_begin,
                  cudaEvent_t main_end) {
  const Grids G = graph_grids<OffT, TB, TT>(g);
  const size_t bm_bytes = sizeof(uint32_t) * (size_t)g->words;
  switch (kase) {
    case 0:
    case 2:
      if (kase == 2) k_bitmap_to_queue<OffT><<<G.conv, kThreads, 0, s>>>(A);
      if (main_begin) cudaEventRecord(main_begin, s);
      k_td_bin<OffT, false, TT><<<G.td_bin, TT, 0, s>>>(A);
      k_td_chunks<OffT, false, TT><<<G.td_chunks, TT, 0, s>>>(A);
      if (main_end) cudaEventRecord(main_end, s);
      break;
    case 1:
    case 3:
      if (kase == 3) {
        DOBFS_CUDA_TRY(cudaMemsetAsync(g->fbm.ptr, 0, 2 * bm_bytes, s));
        k_queue_to_bitmap<OffT><<<G.conv, kThreads, 0, s>>>(A);
      }
      if (main_begin) cudaEventRecord(main_begin, s);
      k_bu<OffT, false, TB><<<G.bu, TB, 0, s>>>(A);
      k_bu_long<OffT><<<G.bu_long, kThreads, 0, s>>>(A);
      if (main_end) cudaEventRecord(main_end, s);
      break;
    case 4:  // top-down with bitmap output, frontier held as a queue
    case 5:  // the same after a bottom-up level (frontier held as a bitmap)
      if (kase == 4) {
        DOBFS_CUDA_TRY(cudaMemsetAsync(g->fbm.ptr, 0, 2 * bm_bytes, s));
        k_queue_to_bitmap<OffT><<<G.conv, kThreads, 0, s>>>(A);
      } else {
        k_bitmap_to_queue<OffT><<<G.conv, kThreads, 0, s>>>(A);
        k_clear_next<OffT><<<G.conv, kThreads, 0, s>>>(A);
      }
      if (main_begin) cudaEventRecord(main_begin, s);
      k_td_bin<OffT, true, TT><<<G.td_bin, TT, 0, s>>>(A);
      k_td_chunks<OffT, true, TT><<<G.td_chunks, TT, 0, s>>>(A);
      k_bu<OffT, false, TB><<<G.bu, TB, 0, s>>>(A);  // the bottom-up part of a mixed level
      k_bu<OffT, true, TB><<<G.bu, TB, 0, s>>>(A);
      k_bu_long<OffT><<<G.bu_long, kThreads, 0, s>>>(A);
      if (main_end) cudaEventRecord(main_end, s);
      break;
    default:
      break;
  }
  DOBFS_CUDA_TRY(cudaGetLastError());
  return DOBFS_OK;
}

template <class OffT, int TB>
int launch_case_td(dobfs_graph* g, const BfsArgs<OffT>& A, int kase, cudaStream_t s, cudaEvent_t mb, cudaEvent_t me,
                   int td) {
  switch (td) {
    case 128: return launch_case_t<OffT, TB, 128>(g, A, kase, s, mb, me);
    case 512: return launch_case_t<OffT, TB, 512>(g, A, kase, s, mb, me);
    default: return launch_case_t<OffT, TB, 256>(g, A, kase, s, mb, me);
  }
}

template <class OffT>
int launch_case(dobfs_graph* g, const BfsArgs<OffT>& A, int kase, cudaStream_t s, cudaEvent_t mb, cudaEvent_t me,
                BlockCfg b) {
  switch (b.bu) {
    case 128: return launch_case_td<OffT, 128>(g, A, kase, s, mb, me, b.td);
    case 512: return launch_case_td<OffT, 512>(g, A, kase, s, mb, me, b.td);
    default: return launch_case_td<OffT, 256>(g, A, kase, s, mb, me, b.td);
  }
}

// The output pass with T threads per block.
template <class OffT, int T>
void launch_output_t(dobfs_graph* g, const BfsArgs<OffT>& A, const int32_t* n2o, int32_t root, int32_t* lv,
                     int32_t* pa, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>(ceil_div(ceil_div(g->n, 4), T), (int64_t)grid_cap(16 * kThreads / T));
  k_output<OffT, T><<<grid, T, 0, s>>>(A, n2o, root, lv, pa);
}

template <class OffT>
void launch_output(dobfs_graph* g, const BfsArgs<OffT>& A, const int32_t* n2o, int32_t root, int32_t* lv,
                   int32_t* pa, cudaStream_t s, int threads) {
  switch (threads) {
    case 128: launch_output_t<OffT, 128>(g, A, n2o, root, lv, pa, s); break;
    case 512: launch_output_t<OffT, 512>(g, A, n2o, root, lv, pa, s); break;
    default: launch_output_t<OffT, 256>(g, A, n2o, root, lv, pa, s); break;
  }
}

template <class OffT>
int build_level_graph(dobfs_graph* g, BlockCfg b) {
  const BfsArgs<OffT> A = make_args<OffT>(g);
  cudaStream_t cs = nullptr;
  DOBFS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  auto fail = [&](int rc) {
    cudaStreamDestroy(cs);
    if (g->cg) cudaGraphDestroy(g->cg);
    g->cg = nullptr;
    return rc;
  };
  if (cudaGraphCreate(&g->cg, 0) != cudaSuccess) return fail(set_error(DOBFS_ERR_CUDA, "cudaGraphCreate failed"));
  cudaGraphConditionalHandle h_while, h_case;
  if (cudaGraphConditionalHandleCreate(&h_while, g->cg, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return fail(set_error(DOBFS_ERR_CUDA, "conditional handle (while) failed"));
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = h_while;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  if (cudaGraphAddNode(&wnode, g->cg, nullptr, nullptr, 0, &wp) != cudaSuccess)
    return fail(set_error(DOBFS_ERR_CUDA, "while node failed: %s", cudaGetErrorString(cudaGetLastError())));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  if (cudaGraphConditionalHandleCreate(&h_case, body, 0, 0) != cudaSuccess)
    return fail(set_error(DOBFS_ERR_CUDA, "conditional handle (switch) failed"));
  // body: the switch kernel ...
  if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return fail(set_error(DOBFS_ERR_CUDA, "capture to body failed"));
  k_switch<OffT><<<1, 32, 0, cs>>>(A, h_while, h_case, 1);
  cudaGraph_t captured = nullptr;
  if (cudaStreamEndCapture(cs, &captured) != cudaSuccess)
    return fail(set_error(DOBFS_ERR_CUDA, "end capture (body) failed"));
  size_t nn = 0;
  cudaGraphGetNodes(body, nullptr, &nn);
  if (nn != 1) return fail(set_error(DOBFS_ERR_CUDA, "unexpected body node count %zu", nn));
  cudaGraphNode_t heur;
  cudaGraphGetNodes(body, &heur, &nn);
  // ... then a switch over the four step kinds
  cudaGraphNodeParams sp = {};
  sp.type = cudaGraphNodeTypeConditional;
  sp.conditional.handle = h_case;
  sp.conditional.type = cudaGraphCondTypeSwitch;
  sp.conditional.size = kCases;
  cudaGraphNode_t snode;
  if (cudaGraphAddNode(&snode, body, &heur, nullptr, 1, &sp) != cudaSuccess)
    return fail(set_error(DOBFS_ERR_CUDA, "switch node failed: %s", cudaGetErrorString(cudaGetLastError())));
  for (int k = 0; k < kCases; ++k) {
    if (cudaStreamBeginCaptureToGraph(cs, sp.conditional.phGraph_out[k], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return fail(set_error(DOBFS_ERR_CUDA, "capture to case %d failed", k));
    int rc = launch_case<OffT>(g, A, k, cs, nullptr, nullptr, b);
    cudaGraph_t cap = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &cap);
    if (rc != DOBFS_OK) return fail(rc);
    if (e != cudaSuccess) return fail(set_error(DOBFS_ERR_CUDA, "end capture case %d: %s", k, cudaGetErrorString(e)));
  }
  cudaError_t e = cudaGraphInstantiate(&g->cg_exec, g->cg, 0);
  if (e != cudaSuccess) return fail(set_error(DOBFS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)));
  cudaStreamDestroy(cs);
  g->cg_bu = b.bu;
  g->cg_td = b.td;
  return DOBFS_OK;
}

// Host-driven levels: same kernels, one round trip per level, every level's
// kernels timed with events (diagnostics).
template <class OffT>
int host_loop(dobfs_graph* g, const BfsArgs<OffT>& A, cudaStream_t s, BlockCfg b) {
  g->host_level_ms.clear();
  g->host_level_main_ms.clear();
  cudaEvent_t e0, e1, m0, m1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventCreate(&m0);
  cudaEventCreate(&m1);
  int rc = DOBFS_OK;
  for (int64_t it = 0; it <= g->n + 1; ++it) {
    k_switch<OffT><<<1, 32, 0, s>>>(A, 0, 0, 0);
    int32_t hdr[8];
    if (cudaMemcpyAsync(hdr, g->ctl.ptr, sizeof(hdr), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = set_error(DOBFS_ERR_CUDA, "host loop: control read failed");
      break;
    }
    const int done = hdr[5], kase = hdr[3];
    if (done) break;
    cudaEventRecord(e0, s);
    rc = launch_case<OffT>(g, A, kase, s, m0, m1, b);
    cudaEventRecord(e1, s);
    if (rc != DOBFS_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0.f, mm = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventElapsedTime(&mm, m0, m1);
    g->host_level_ms.push_back(ms);
    g->host_level_main_ms.push_back(mm);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(m0);
  cudaEventDestroy(m1);
  return rc;
}

template <class OffT>
int run_impl(dobfs_graph* g, int32_t root, int32_t* level_out, int32_t* parent_out, const dobfs_run_opts& o,
             dobfs_run_stats* stats) {
  cudaStream_t s = (cudaStream_t)o.stream;
  if (!s) s = g->stream;
  const bool host_loop_mode = (o.flags & DOBFS_RUN_HOST_LOOP) != 0;
  const bool want_stats = stats || (o.flags & DOBFS_RUN_SYNC_STATS) || kBoundsCheck;
  const bool dev_level = is_device_ptr(level_out);
  const bool dev_parent = parent_out ? is_device_ptr(parent_out) : dev_level;
  if (dev_level != dev_parent)
    return set_error(DOBFS_ERR_INVALID, "level_out and parent_out must both be host or both be device memory");
  if (g->last_stream && g->last_stream != s) DOBFS_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_done, 0));
  const BlockCfg bc = block_cfg(o);
  // small graphs (and default block sizes): one cooperative launch for all levels
  const int fused_grid = (!host_loop_mode && !(o.flags & DOBFS_RUN_LEVEL_GRAPH) && !g->fused_off &&
                          bc.bu == kThreads && bc.td == kThreads)
                             ? fused_grid_for<OffT>(g)
                             : 0;
  bool fused = fused_grid > 0;
  // the level graph for this run's block sizes
  auto ensure_level_graph = [&]() -> int {
    if (g->cg_exec && (g->cg_bu != bc.bu || g->cg_td != bc.td)) {
      // another block configuration: the level graph is rebuilt for it
      // (after the previous run, which may still use the old one)
      DOBFS_CUDA_TRY(cudaEventSynchronize(g->ev_done));
      cudaGraphExecDestroy(g->cg_exec);
      cudaGraphDestroy(g->cg);
      g->cg_exec = nullptr;
      g->cg = nullptr;
    }
    if (!g->cg_exec) DOBFS_TRY(build_level_graph<OffT>(g, bc));
    return DOBFS_OK;
  };
  if (!host_loop_mode && !fused) DOBFS_TRY(ensure_level_graph());
  const BfsArgs<OffT> A = make_args<OffT>(g);
  int32_t* lv = level_out;
  int32_t* pa = parent_out;
  if (!dev_level) {
    if (!g->out_stage.ptr) DOBFS_TRY(g->out_stage.alloc(sizeof(int32_t) * 2 * (size_t)g->n, g->stream));
    lv = g->out_stage.as<int32_t>();
    pa = parent_out ? lv + g->n : nullptr;
  }
  RunParams P;
  P.root_orig = root;
  P.mode = o.direction;
  P.alpha = o.alpha;
  P.beta = o.beta;
  P.static_pct = o.static_pct;
  P.bu_steps = o.bu_steps;
  P.sched_seed = o.schedule_seed;
  P.td_bm_div = o.td_bitmap_div;
  P.td_small = o.td_small_max ? o.td_small_max : kTdSmall;
  P.td_chunk = o.td_chunk ? o.td_chunk : kChunk;
  P.bu_scan = o.bu_scan ? o.bu_scan : kBuT;
  P.td_split_pct = o.td_split_pct;
  DOBFS_CUDA_TRY(cudaEventRecord(g->ev_t0, s));
  if (fused) {
    // the whole level loop, status init included, in one cooperative launch
    void* args[] = {(void*)&A, (void*)&P};
    const cudaError_t e =
        cudaLaunchCooperativeKernel((const void*)k_bfs_fused<OffT>, dim3(fused_grid), dim3(kThreads), args, 0, s);
    if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported || e == cudaErrorNotPermitted) {
      // this context cannot hold the grid at once (a partitioned or shared
      // device, say): nothing was launched; the level graph runs this BFS
      // and the graph's later ones
      cudaGetLastError();
      g->fused_off = true;
      fused = false;
      DOBFS_TRY(ensure_level_graph());
    } else {
      DOBFS_CUDA_TRY(e);
    }
  }
  if (!fused) {
    DOBFS_CUDA_TRY(cudaMemsetAsync(g->visited.ptr, 0, sizeof(uint32_t) * (size_t)g->words, s));
    k_init<OffT><<<1, 32, 0, s>>>(A, P);
    DOBFS_CUDA_TRY(cudaGetLastError());
    if (host_loop_mode) {
      DOBFS_TRY(host_loop<OffT>(g, A, s, bc));
    } else {
      DOBFS_CUDA_TRY(cudaGraphLaunch(g->cg_exec, s));
    }
  }
  const int32_t* n2o = g->reindexed ? g->new2orig.as<int32_t>() : nullptr;
  launch_output<OffT>(g, A, n2o, root, lv, pa, s, o.out_threads ? o.out_threads : kThreads);
  if (pa && (o.flags & DOBFS_RUN_CANONICAL_PARENT))
    k_canonical_parent<OffT><<<grid_cap(8), kThreads, 0, s>>>(A, n2o, pa);
  DOBFS_CUDA_TRY(cudaGetLastError());
  if (!dev_level) {
    DOBFS_CUDA_TRY(cudaMemcpyAsync(level_out, lv, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, s));
    if (parent_out)
      DOBFS_CUDA_TRY(cudaMemcpyAsync(parent_out, pa, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, s));
  }
  DOBFS_CUDA_TRY(cudaEventRecord(g->ev_t1, s));
  DOBFS_CUDA_TRY(cudaEventRecord(g->ev_done, s));
  g->last_stream = s;
  g->last_host_loop = host_loop_mode;
  g->last_trace_batch = false;
  if (!dev_level) DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  if (want_stats) {
    DOBFS_CUDA_TRY(cudaEventSynchronize(g->ev_t1));
    BfsCtl c;
    DOBFS_CUDA_TRY(cudaMemcpy(&c, g->ctl.ptr, sizeof(c), cudaMemcpyDeviceToHost));
    if (c.bc_site)
      return set_error(DOBFS_ERR_BOUNDS, "device bounds check failed: %s", bounds_site_name(c.bc_site));
    if (c.overflow == 2) return set_error(DOBFS_ERR_CUDA, "internal: the level loop ran past n levels");
    if (c.overflow == 3) return set_error(DOBFS_ERR_CUDA, "internal: a grid barrier of the fused level loop timed out");
    if (c.overflow) return set_error(DOBFS_ERR_CUDA, "internal: top-down record buffer overflow");
    if (stats) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, g->ev_t0, g->ev_t1);
      stats->device_ms = ms;
      stats->levels = c.n_levels;
      stats->td_levels = c.n_td;
      stats->bu_levels = c.n_bu;
      stats->reached = c.reached;
      stats->teps_edges = c.teps2 / 2;
      stats->edges_examined = c.examined;
      // output pass: 8 bytes written per vertex, the map read when renumbered,
      // and the (level, parent) pair of every reached vertex
      stats->alg_bytes = c.alg_bytes + 8 * g->n + (g->reindexed ? 4 * g->n : 0) + 8 * c.reached;
    }
  }
  return DOBFS_OK;
}

}  // namespace

int graph_alloc_workspace(dobfs_graph* g) {
  cudaStream_t s = g->stream;
  const size_t wb = sizeof(uint32_t) * (size_t)g->words;
  DOBFS_TRY(g->visited.alloc(wb, s));
  DOBFS_TRY(g->fbm.alloc(2 * wb, s));
  DOBFS_CUDA_TRY(cudaMemsetAsync(g->fbm.ptr, 0, 2 * wb, s));
  DOBFS_TRY(g->lp.alloc(sizeof(int2) * (size_t)g->n, s));
  DOBFS_TRY(g->q0.alloc(sizeof(int32_t) * (size_t)g->n, s));
  DOBFS_TRY(g->q1.alloc(sizeof(int32_t) * (size_t)g->n, s));
  g->rec_cap = std::min<int64_t>(g->n, g->nnz / (kTdSmallMin + 1)) + g->nnz / kChunkMin + 64;
  DOBFS_TRY(g->rec.alloc(sizeof(int2) * (size_t)g->rec_cap, s));
  DOBFS_TRY(g->deferred.alloc(sizeof(int32_t) * (size_t)g->n, s));
  DOBFS_TRY(g->firstdeg.alloc(sizeof(int2) * (size_t)g->n, s));
  DOBFS_TRY(g->degge.alloc(sizeof(g->deg_ge) + sizeof(g->small_tab), s));
  DOBFS_CUDA_TRY(cudaMemcpyAsync(g->degge.ptr, g->deg_ge, sizeof(g->deg_ge), cudaMemcpyHostToDevice, s));
  DOBFS_CUDA_TRY(cudaMemcpyAsync(g->degge.as<int64_t>() + 33, g->small_tab, sizeof(g->small_tab),
                                 cudaMemcpyHostToDevice, s));
  {
    const int grid = (int)std::min<int64_t>(ceil_div(g->n, kThreads), (int64_t)grid_cap(16));
    if (g->off64)
      k_firstdeg<int64_t><<<grid, kThreads, 0, s>>>(g->off.as<int64_t>(), g->cols.as<int32_t>(), g->n,
                                                   g->firstdeg.as<int2>());
    else
      k_firstdeg<int32_t><<<grid, kThreads, 0, s>>>(g->off.as<int32_t>(), g->cols.as<int32_t>(), g->n,
                                                   g->firstdeg.as<int2>());
    DOBFS_CUDA_TRY(cudaGetLastError());
  }
  // the control block, then the fused loop's grid barrier (4 words)
  DOBFS_TRY(g->ctl.alloc(sizeof(BfsCtl) + kGridBarBytes, s));
  DOBFS_TRY(g->trace.alloc(sizeof(LevelRec) * kMaxTrace, s));
  DOBFS_CUDA_TRY(cudaMemsetAsync(g->ctl.ptr, 0, sizeof(BfsCtl) + kGridBarBytes, s));
  DOBFS_CUDA_TRY(cudaEventCreate(&g->ev_done));
  DOBFS_CUDA_TRY(cudaEventCreate(&g->ev_t0));
  DOBFS_CUDA_TRY(cudaEventCreate(&g->ev_t1));
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  g->ws_ready = true;
  return DOBFS_OK;
}

int graph_levels_async(dobfs_graph* g, int32_t* dst, cudaStream_t s) {
  DOBFS_CUDA_TRY(cudaMemcpyAsync(dst, &g->ctl.as<BfsCtl>()->n_levels, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  return DOBFS_OK;
}

void graph_release(dobfs_graph* g) {
  // wait through the graph's own event: the stream of the last run may no
  // longer exist (a caller's or the server's stream)
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->ev_done) cudaEventSynchronize(g->ev_done);
  g->last_stream = nullptr;
  ms_group_destroy(g->ms);
  g->ms = nullptr;
  for (int k = 0; k < kMsConcurrent - 1; ++k) {
    ms_group_destroy(g->ms_more[k]);
    g->ms_more[k] = nullptr;
    if (g->ms_streams[k]) cudaStreamDestroy(g->ms_streams[k]);
    if (g->ms_ev_join[k]) cudaEventDestroy(g->ms_ev_join[k]);
    g->ms_streams[k] = nullptr;
    g->ms_ev_join[k] = nullptr;
  }
  if (g->ms_ev_fork) cudaEventDestroy(g->ms_ev_fork);
  g->ms_ev_fork = nullptr;
  if (g->cg_exec) cudaGraphExecDestroy(g->cg_exec);
  if (g->cg) cudaGraphDestroy(g->cg);
  g->cg_exec = nullptr;
  g->cg = nullptr;
  if (g->ev_done) cudaEventDestroy(g->ev_done);
  if (g->ev_t0) cudaEventDestroy(g->ev_t0);
  if (g->ev_t1) cudaEventDestroy(g->ev_t1);
  g->ev_done = g->ev_t0 = g->ev_t1 = nullptr;
}

}  // namespace dobfs

using namespace dobfs;

extern "C" {

int dobfs_run_opts_init(dobfs_run_opts* o) {
  if (!o) return set_error(DOBFS_ERR_INVALID, "opts is NULL");
  o->direction = DOBFS_DIR_AUTO;
  o->alpha = 14;
  o->beta = 24;
  o->static_pct = 10;
  o->bu_steps = 3;
  o->flags = 0;
  o->schedule_seed = 0;
  o->stream = nullptr;
  o->td_bitmap_div = 2;
  o->td_small_max = 0;
  o->td_chunk = 0;
  o->bu_scan = 0;
  o->td_split_pct = 150;
  o->bu_threads = 0;
  o->td_threads = 0;
  o->out_threads = 0;
  return DOBFS_OK;
}

int dobfs_run(dobfs_graph* g, int32_t root, int32_t* level_out, int32_t* parent_out, const dobfs_run_opts* opts,
              dobfs_run_stats* stats) {
  clear_error();
  if (!g || !level_out) return set_error(DOBFS_ERR_INVALID, "graph and level_out are required");
  if (root < 0 || (int64_t)root >= g->n)
    return set_error(DOBFS_ERR_INVALID, "root %d out of range [0, %lld)", root, (long long)g->n);
  dobfs_run_opts o;
  dobfs_run_opts_init(&o);
  if (opts) o = *opts;
  if (o.direction < 0 || o.direction > DOBFS_DIR_STATIC || o.alpha < 1 || o.beta < 1 || o.static_pct < 0 ||
      o.bu_steps < 1 || o.td_bitmap_div < 0)
    return set_error(DOBFS_ERR_INVALID, "bad run options");
  if (!cutoffs_valid(o)) return set_error(DOBFS_ERR_INVALID, "bad degree-bin cutoffs");
  std::lock_guard<std::mutex> lk(g->mu);
  return g->off64 ? run_impl<int64_t>(g, root, level_out, parent_out, o, stats)
                  : run_impl<int32_t>(g, root, level_out, parent_out, o, stats);
}

int dobfs_last_trace(const dobfs_graph* gc, dobfs_level_trace* out, int32_t max_levels, int32_t* n_out) {
  if (!gc || !out || !n_out || max_levels < 0) return set_error(DOBFS_ERR_INVALID, "bad trace arguments");
  dobfs_graph* g = const_cast<dobfs_graph*>(gc);
  std::lock_guard<std::mutex> lk(g->mu);
  DOBFS_CUDA_TRY(cudaEventSynchronize(g->ev_done));
  if (g->last_trace_batch) {
    const int32_t nb = (int32_t)std::min<size_t>(g->batch_trace.size(), (size_t)max_levels);
    for (int32_t i = 0; i < nb; ++i) out[i] = g->batch_trace[i];
    *n_out = nb;
    return DOBFS_OK;
  }
  BfsCtl c;
  DOBFS_CUDA_TRY(cudaMemcpy(&c, g->ctl.ptr, sizeof(c), cudaMemcpyDeviceToHost));
  const int32_t n = std::min<int32_t>(std::min<int32_t>(c.n_levels, kMaxTrace), max_levels);
  std::vector<LevelRec> rec((size_t)std::max(n, 0));
  if (n > 0) DOBFS_CUDA_TRY(cudaMemcpy(rec.data(), g->trace.ptr, sizeof(LevelRec) * (size_t)n, cudaMemcpyDeviceToHost));
  for (int32_t i = 0; i < n; ++i) {
    out[i].level = rec[i].level;
    out[i].direction = rec[i].dir;
    out[i].n_frontier = rec[i].n_f;
    out[i].m_frontier = rec[i].m_f;
    out[i].m_unvisited = rec[i].m_u;
    out[i].n_next = rec[i].n_next;
    out[i].edges_examined = rec[i].examined;
    out[i].vertices_scanned = rec[i].scanned;
    out[i].alg_bytes = rec[i].bytes;
    const bool timed = g->last_host_loop && (size_t)i < g->host_level_ms.size();
    out[i].ms = timed ? g->host_level_ms[i] : 0.f;
    out[i].ms_main = timed ? g->host_level_main_ms[i] : 0.f;
  }
  *n_out = n;
  return DOBFS_OK;
}

int dobfs_graph_destroy(dobfs_graph* g) {
  if (!g) return DOBFS_OK;
  {
    std::lock_guard<std::mutex> lk(g->mu);
    graph_release(g);
  }
  delete g;
  return DOBFS_OK;
}

int dobfs_debug_set_column(dobfs_graph* g, int64_t pos, int32_t value) {
  clear_error();
  if (!kBoundsCheck) return set_error(DOBFS_ERR_INVALID, "dobfs_debug_set_column: bounds-check builds only");
  if (!g) return set_error(DOBFS_ERR_INVALID, "graph is NULL");
  if (pos < 0 || pos >= g->nnz)
    return set_error(DOBFS_ERR_INVALID, "entry %lld out of range [0, %lld)", (long long)pos, (long long)g->nnz);
  if (value < 0 || (int64_t)value >= g->n + kBoundsSlackVertices)
    return set_error(DOBFS_ERR_INVALID, "value %d outside [0, n + %lld)", value, (long long)kBoundsSlackVertices);
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t s = g->stream;
  if (g->last_stream) DOBFS_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_done, 0));
  DOBFS_CUDA_TRY(cudaMemcpyAsync(g->cols.as<int32_t>() + pos, &value, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  const int grid = (int)std::min<int64_t>(ceil_div(g->n, kThreads), (int64_t)grid_cap(16));
  if (g->off64)
    k_firstdeg<int64_t><<<grid, kThreads, 0, s>>>(g->off.as<int64_t>(), g->cols.as<int32_t>(), g->n,
                                                 g->firstdeg.as<int2>());
  else
    k_firstdeg<int32_t><<<grid, kThreads, 0, s>>>(g->off.as<int32_t>(), g->cols.as<int32_t>(), g->n,
                                                 g->firstdeg.as<int2>());
  DOBFS_CUDA_TRY(cudaGetLastError());
  DOBFS_CUDA_TRY(cudaStreamSynchronize(s));
  return DOBFS_OK;
}

int dobfs_debug_grid_barrier(int32_t blocks, int32_t rounds, int32_t missing, int32_t* rounds_passed,
                             int32_t* short_counts, int32_t* timed_out) {
  clear_error();
  if (!rounds_passed || !short_counts || !timed_out) return set_error(DOBFS_ERR_INVALID, "output pointers are NULL");
  int per_sm = 0;
  DOBFS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_probe, kThreads, 0));
  const int64_t cap = (int64_t)sm_count() * per_sm;
  if (blocks < 1 || blocks > cap || rounds < 0 || rounds > (1 << 20) || missing < 0 || missing > 1)
    return set_error(DOBFS_ERR_INVALID, "bad barrier test: blocks %d (1..%lld), rounds %d, missing %d", blocks,
                     (long long)cap, rounds, missing);
  DevBuf buf;  // barrier words (4), then the counters (4)
  DOBFS_TRY(buf.alloc(8 * sizeof(uint32_t), nullptr));
  uint32_t* bar = buf.as<uint32_t>();
  uint32_t* cnt = bar + 4;
  DOBFS_CUDA_TRY(cudaMemsetAsync(bar, 0, 8 * sizeof(uint32_t), nullptr));
  uint32_t r = (uint32_t)rounds, m = (uint32_t)missing;
  void* args[] = {(void*)&bar, (void*)&cnt, (void*)&r, (void*)&m};
  DOBFS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_barrier_probe, dim3(blocks), dim3(kThreads), args, 0,
                                             nullptr));
  uint32_t h[8];
  DOBFS_CUDA_TRY(cudaMemcpy(h, bar, sizeof(h), cudaMemcpyDeviceToHost));
  *rounds_passed = (int32_t)h[5];
  *short_counts = (int32_t)h[6];
  *timed_out = (int32_t)(h[2] != 0);
  return DOBFS_OK;
}

}  // extern "C"
