// Bit-parallel multi-source BFS (64 or 128 roots per lane group) on a dobfs_graph.
//
// Used by dobfs_run_batch (a group runs a batch of up to 128 roots to the end)
// and by the query server (lanes join and leave a running group at level
// boundaries). A group owns its per-vertex lane masks and its control block;
// the graph's CSR is shared read-only.
#pragma once

#include "common.cuh"
#include "graph.cuh"

namespace dobfs {

constexpr int kMsWordLanes = 64;                 // lanes per 64-bit mask word
constexpr int kMsMaxWords = 2;                   // mask words per vertex: 64 or 128 lanes per group
constexpr int kMsLanes = kMsWordLanes * kMsMaxWords;  // most lanes of a group
constexpr int kMsPlanes = 16;  // discovery iterations are kept mod 2^16

// Host-side set of up to kMsLanes lanes (bit l = lane l).
using LaneMask = unsigned __int128;
inline LaneMask lane_bit(int l) { return (LaneMask)1 << l; }
inline uint64_t lane_word(LaneMask m, int w) { return (uint64_t)(m >> (kMsWordLanes * w)); }
inline LaneMask lanes_of(const unsigned long long* words, int n_words) {
  LaneMask m = 0;
  for (int w = 0; w < n_words; ++w) m |= (LaneMask)words[w] << (kMsWordLanes * w);
  return m;
}
inline int first_lane(LaneMask m) {  // m != 0
  const uint64_t lo = (uint64_t)m;
  return lo ? __builtin_ctzll(lo) : kMsWordLanes + __builtin_ctzll((uint64_t)(m >> kMsWordLanes));
}

// Per-lane frontier statistics of a lane group, sampled from every
// kMsLaneSample-th block of 32 vertices (estimates; they choose directions
// only, never results): vertices in the lane's frontier, their degree sum,
// the degree sum of the vertices the lane has not reached.
constexpr int kMsLaneSample = 64;
struct MsLaneStats {
  unsigned long long n_f[kMsLanes], m_f[kMsLanes], m_u[kMsLanes];
  unsigned long long n_f_prev[kMsLanes];
};

// Device control block of a lane group.
struct MsCtl {
  int32_t iter;          // iteration t: the frontier holds the vertices found at iteration t
  int32_t dir;           // direction of the step expanding iteration t: 0 top-down, 1 bottom-up
  int32_t step_case;
  int32_t fresh;
  int32_t done;
  int32_t n_planes;      // planes cleared so far (planes >= n_planes hold stale bits)
  int32_t clear_plane;   // plane the running step clears first (-1: none)
  int32_t levels_run;    // steps since the last reset
  unsigned long long active[kMsMaxWords];  // lanes holding a query
  unsigned long long live[kMsMaxWords];    // lanes with a non-empty frontier
  int64_t n_f, m_f, m_u, n_f_prev;
  // accumulators of the running step
  unsigned long long nx_n, nx_m, nx_mu, nx_examined;
  unsigned long long nx_act;   // bottom-up: vertices still missing live lanes (searched)
  unsigned long long nx_tdact; // top-down: frontier vertices whose rows were pushed
  // directions by lane: the running step expands the lanes of td_mask
  // top-down and those of bu_mask bottom-up (step_case 2 when both are
  // non-empty); lane_bu holds the lanes whose last step was bottom-up
  unsigned long long td_mask[kMsMaxWords], bu_mask[kMsMaxWords], lane_bu[kMsMaxWords];
  unsigned long long nx_live[kMsMaxWords];
  unsigned int n_rec, n_def;
  // parameters
  int32_t mode, alpha, beta, td_chunk, bu_scan;  // policy and degree-bin cutoffs
  int32_t bc_site;       // bounds-check builds: first failing check (0: none)
  int32_t runaway;       // graph-driven loop stopped after n iterations (a fault; never expected)
  uint64_t sched_seed;
  int64_t examined;
  // algorithmic DRAM bytes of the steps since the last reset: per step,
  // 16 W per active vertex (its seen and next masks of W 8-byte words; a
  // top-down step's active vertices are its frontier, a bottom-up step's the
  // vertices it searches) + (8 W + 4) per examined entry (the neighbour's
  // frontier mask and the column)
  int64_t alg_bytes;
};

struct MsGroup {
  dobfs_graph* g = nullptr;
  cudaStream_t stream = nullptr;
  int words = 1;          // mask words per vertex: lanes = 64 * words
  // per vertex v, words [v * words, (v + 1) * words) of each mask array
  DevBuf seen, fb0, fb1;  // uint64[n][words]: lanes that reached v; frontier masks by iteration parity
  DevBuf planes;          // uint64[kMsPlanes][n][words]: bit b of the discovery iteration, per lane
  DevBuf rec;             // int2[]: top-down chunk records
  int64_t rec_cap = 0;
  DevBuf def;             // int32[n]: bottom-up rows continued warp-wide
  DevBuf ctl;             // MsCtl
  DevBuf lstats;          // MsLaneStats
  DevBuf args;            // device copy of seeding arguments
  cudaGraph_t cg = nullptr;
  cudaGraphExec_t exec = nullptr;
  int bu_threads = 256, td_threads = 256;  // block sizes of the step's main kernels (set by a reset)
  int graph_bu = 0, graph_td = 0;          // block sizes the loop graph was built with
};

// Device bytes of one lane group of `words` mask words on g (what ms_group_create allocates).
int64_t ms_group_bytes(const dobfs_graph* g, int words);
// Creates a group of 64 * words lanes (words 1 or 2) on g (allocates its
// masks); *out owned by the caller.
int ms_group_create(dobfs_graph* g, cudaStream_t s, int words, MsGroup** out);
void ms_group_destroy(MsGroup* m);

// Clears every mask and counter (all lanes free).
int ms_group_reset(MsGroup* m, const dobfs_run_opts& o);

// Starts lanes lane[i] at the current iteration from original-ID roots root[i].
int ms_group_seed(MsGroup* m, int count, const int32_t* lane, const int32_t* root);

// One level from the host (the server's loop) or the whole loop as one graph launch.
// after_switch / case_ms (nullable) receive the control block after the
// direction switch and the device time of the step's kernels.
int ms_group_step(MsGroup* m, MsCtl* after_switch, float* case_ms);
int ms_group_run_to_end(MsGroup* m);

// Writes levels of the lanes in `lanes` into out[i][n] (original IDs; -1 if
// unreached), levels counted from start[i]; with `release` the lanes' bits
// are cleared and the lanes freed.
int ms_group_flush(MsGroup* m, LaneMask lanes, int32_t* const* out, const int32_t* start, bool release);

// Server loop pieces, all asynchronous on the group's stream: the direction
// switch followed by a copy of the control block into `dst` (pinned host
// memory), and the kernels of one step (0 top-down, 1 bottom-up, 2 both:
// some lanes top-down, the others bottom-up).
int ms_group_switch_async(MsGroup* m, MsCtl* dst);
int ms_group_case_async(MsGroup* m, int kase);

// Reads the control block (synchronises the group's stream).
int ms_group_read_ctl(MsGroup* m, MsCtl* c);
// Iteration count back to 0 once no lane holds a query (on the group's stream).
int ms_group_rebase(MsGroup* m);

}  // namespace dobfs
