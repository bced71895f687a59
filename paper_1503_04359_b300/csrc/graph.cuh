// The graph object behind the dobfs_graph handle: the stored CSR (device),
// the renumbering maps, and the per-graph BFS workspace.
#pragma once

#include <mutex>
#include <vector>

#include "common.cuh"

namespace dobfs {

struct MsGroup;

// Lane groups of one batch that run at the same time (on as many streams).
constexpr int kMsConcurrent = 4;

// Sentinel edge key: a dropped entry (self-loop or duplicate). Sorts last.
constexpr uint64_t kSentinelKey = ~0ull;

// Degrees below kSmallDeg are classes of their own in the renumbering, so a
// row of such a vertex starts at an offset computed from its ID.
constexpr int kSmallDeg = 8;

// Degree-bin cutoffs of a run: 0 (the path's default) or within the ranges
// the record buffers are sized for.
inline bool cutoffs_valid(const dobfs_run_opts& o) {
  const bool small_ok = o.td_small_max == 0 || (o.td_small_max >= 8 && o.td_small_max <= 256);
  const bool chunk_ok = o.td_chunk == 0 || (o.td_chunk >= 256 && o.td_chunk <= 8192 && o.td_chunk % 128 == 0);
  const bool scan_ok = o.bu_scan == 0 || (o.bu_scan >= 1 && o.bu_scan <= 256);
  const bool split_ok = o.td_split_pct >= 0 && o.td_split_pct <= 100000;
  auto block_ok = [](int32_t t) { return t == 0 || t == 128 || t == 256 || t == 512; };
  const bool blocks_ok = block_ok(o.bu_threads) && block_ok(o.td_threads) && block_ok(o.out_threads);
  return small_ok && chunk_ok && scan_ok && split_ok && blocks_ok;
}

// Device-side control block of one BFS run (one per graph). The level loop
// reads and updates it on the device; the host reads it only after a run.
struct BfsCtl {
  int32_t level;        // L: the frontier holds the vertices at level L
  int32_t dir;          // direction of the step expanding level L: 0 top-down, 1 bottom-up
  int32_t fmt;          // frontier of level L is held as 0: queue, 1: bitmap
  int32_t step_case;    // 0 TD from queue, 1 BU from bitmap, 2 TD after bitmap->queue, 3 BU after queue->bitmap,
                        // 4/5 TD with bitmap output (from queue / from bitmap)
  int32_t fresh;        // set by init: the loop has not run a step yet
  int32_t done;
  int32_t bu_run;       // consecutive bottom-up levels so far (static policy)
  int32_t n_levels;
  int64_t n_f, m_f;     // size and degree sum of the level-L frontier
  int64_t n_f_prev;
  int64_t m_u;          // degree sum of vertices not yet visited
  // accumulators of the running step, reset by the heuristic kernel
  unsigned long long nx_n, nx_m, nx_examined, nx_scanned;
  unsigned int q_tail;  // next-queue tail (top-down) / bitmap->queue tail
  unsigned int n_rec;   // top-down chunk records
  unsigned int n_def;   // bottom-up deferred (long) rows
  unsigned int conv_tail;  // bitmap->queue conversion tail
  unsigned int out_next;   // output pass: next chunk of original IDs to take
  // run totals
  int64_t reached, teps2, examined, alg_bytes;
  int32_t n_td, n_bu;
  int32_t overflow;     // top-down record buffer overflow (never expected)
  int32_t bc_site;      // bounds-check builds: first failing check (0: none)
  // parameters
  int32_t mode, alpha, beta, static_pct, bu_steps, td_bm_div;
  int32_t td_small, td_chunk, bu_scan, td_split_pct;  // degree-bin cutoffs; mixed-level threshold
  int64_t split_w;      // mixed level: words [0, split_w) bottom-up, targets beyond them top-down (0: none)
  uint64_t sched_seed;
};

// Per-level trace record on the device (mirrors dobfs_level_trace).
struct LevelRec {
  int32_t level, dir;
  int64_t n_f, m_f, m_u, n_next, examined, scanned, bytes;
};
constexpr int kMaxTrace = 4096;

}  // namespace dobfs

struct dobfs_graph {
  int64_t n = 0;            // vertices
  int64_t nnz = 0;          // stored directed entries
  int64_t n_nonisolated = 0;
  int64_t max_degree = 0;
  int bits = 0;             // bits per vertex ID in edge keys
  bool off64 = false;
  bool reindexed = false;
  float build_ms = 0.f;
  cudaStream_t stream = nullptr;

  // stored CSR (internal IDs). cols carries 4 padding entries so 16-byte
  // vector loads of a row's last aligned chunk stay inside the allocation.
  dobfs::DevBuf off, cols;
  dobfs::DevBuf new2orig, orig2new;  // int32[n] each, only when reindexed
  dobfs::DevBuf isolated;            // bitmap: degree-0 vertices and bits >= n
  int64_t deg_ge[33] = {};           // vertices of degree >= 2^k (a prefix of the IDs when reindexed)
  // renumbered graphs: [d] row offset and [kSmallDeg + d] first ID of the
  // vertices of degree d, for 1 <= d < small_deg (small_deg = 0: not used)
  int64_t small_tab[2 * dobfs::kSmallDeg] = {};
  int32_t small_deg = 0;
  int64_t words = 0;                 // bitmap words = ceil(n/32)

  // BFS workspace
  dobfs::DevBuf visited;              // bitmap
  dobfs::DevBuf fbm;                  // both frontier bitmaps: words [0, words) and [words, 2 words)
  dobfs::DevBuf lp;                   // int2[n]: (level, parent) in internal IDs
  dobfs::DevBuf q0, q1;               // int32[n] queues
  dobfs::DevBuf rec;                  // int2[] top-down chunk records
  int64_t rec_cap = 0;
  dobfs::DevBuf deferred;             // int32[n]
  dobfs::DevBuf firstdeg;             // int2[n]: (first neighbour, degree)
  dobfs::DevBuf degge;                // int64[33 + 2 * kSmallDeg]: device copy of deg_ge, small_tab
  dobfs::DevBuf ctl;                  // BfsCtl
  dobfs::DevBuf trace;                // LevelRec[kMaxTrace]
  dobfs::DevBuf out_stage;            // int32[2n] staging for host outputs (lazy)
  bool ws_ready = false;

  // level loop as a CUDA graph with a device-driven while node
  cudaGraph_t cg = nullptr;
  cudaGraphExec_t cg_exec = nullptr;
  int cg_bu = 0, cg_td = 0;           // block sizes the level graph was built with
  bool fused_off = false;             // a cooperative launch was refused here: level graph only
  cudaEvent_t ev_done = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  cudaStream_t last_stream = nullptr;
  bool last_host_loop = false;
  std::vector<float> host_level_ms, host_level_main_ms;

  // batched runs: one lane group and a staging buffer for host outputs
  dobfs::MsGroup* ms = nullptr;
  // more groups, so that the groups of a batch overlap, each further one on
  // its own stream
  dobfs::MsGroup* ms_more[dobfs::kMsConcurrent - 1] = {};
  cudaStream_t ms_streams[dobfs::kMsConcurrent - 1] = {};
  cudaEvent_t ms_ev_fork = nullptr;
  cudaEvent_t ms_ev_join[dobfs::kMsConcurrent - 1] = {};
  dobfs::DevBuf ms_stage;
  std::vector<dobfs_level_trace> batch_trace;  // host-driven batch levels (first group)
  bool last_trace_batch = false;

  std::mutex mu;
};

namespace dobfs {

int graph_alloc_workspace(dobfs_graph* g);
// Copies the level count of the last single-source run on g to dst (pinned host memory), on s.
int graph_levels_async(dobfs_graph* g, int32_t* dst, cudaStream_t s);
void graph_release(dobfs_graph* g);

// builds g's CSR from n_keys edge keys (row<<bits | col, or kSentinelKey),
// consuming `keys` (n_keys entries, may be reordered/overwritten)
int build_from_keys(dobfs_graph* g, DevBuf& keys, int64_t n_keys, uint32_t flags, cudaStream_t s);

// A new empty graph of n vertices (DOBFS_ERR_INVALID unless 1 <= n < 2^31).
int new_graph(int64_t n, cudaStream_t s, dobfs_graph** out);
// Events timing a build on s (e0 recorded now).
int start_timer(cudaStream_t s, cudaEvent_t* e0, cudaEvent_t* e1);
// Ends a build with status rc: on success allocates the BFS workspace and
// hands g to *out; on failure releases g and sets *out = NULL.
int finish_graph(dobfs_graph* g, int rc, cudaEvent_t e0, cudaEvent_t e1, dobfs_graph** out);
// Reads a device error flag written on s.
int read_err_flag(DevBuf& err, cudaStream_t s, int* h);
// Takes over a stored CSR placed in g->off / g->cols (and g->new2orig when
// g->reindexed; g->orig2new allocated): checks the build's invariants
// (DOBFS_ERR_BAD_GRAPH otherwise), fills orig2new and the degree statistics.
int adopt_csr(dobfs_graph* g, bool check_symmetric, cudaStream_t s);

}  // namespace dobfs
