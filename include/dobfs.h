/*
 * dobfs — direction-optimized breadth-first search on one GPU (C ABI).
 *
 * The method is the per-level step of direction-optimized BFS (Sec. 2.2 and
 * Algorithm 1 of Sallinen, Gharaibeh & Ripeanu, "Accelerating Direction-
 * Optimized Breadth First Search on Hybrid Architectures"): a level is
 * expanded either top-down (every frontier vertex marks its unvisited
 * neighbours, Algorithm 1 top-down branch) or bottom-up (every unvisited
 * vertex looks for a neighbour in the frontier and stops at the first one,
 * Algorithm 1 bottom-up branch), and the direction switches between the two
 * from frontier vertex and edge counts (Sec. 3.3). Here the whole graph lives
 * in one GPU's memory; every step runs in this library's CUDA kernels and
 * the direction is chosen on the device, so a level needs no host round trip.
 *
 * Conventions
 *  - Every function returns a dobfs_status; nothing throws or aborts across
 *    this boundary. dobfs_last_error() describes the last failure of the
 *    calling thread.
 *  - Vertex IDs at this boundary are the caller's IDs ("original IDs"),
 *    int32 in [0, n_vertices). A graph built with DOBFS_GRAPH_REINDEX
 *    renumbers vertices internally; outputs are always in original IDs.
 *  - Output conventions (the paper states none): an unreached vertex has
 *    level -1 and parent -1; level[root] = 0 and parent[root] = root.
 *  - Pointers are host or device pointers; the library tells them apart with
 *    cudaPointerGetAttributes unless a flag says otherwise. Caller memory is
 *    never freed by the library. Input arrays are copied; output arrays must
 *    stay valid until the call (or, for the server, the poll) has completed.
 *  - `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *    legacy default stream). Calls on one graph are serialised by the
 *    library: a run on another stream first waits for the previous run.
 */
#ifndef DOBFS_H
#define DOBFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DOBFS_OK = 0,
  DOBFS_PENDING = 1,          /* server query not finished yet */
  DOBFS_ERR_INVALID = -1,     /* bad argument (NULL handle, root out of range, size < 0, ...) */
  DOBFS_ERR_OOM = -2,         /* device allocation failed */
  DOBFS_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  DOBFS_ERR_BAD_GRAPH = -4,   /* column out of range, or asymmetric input under VALIDATE */
  DOBFS_ERR_TIMEOUT = -5,     /* a bounded host wait ran out (dobfs_graph_wait) */
  DOBFS_ERR_BUSY = -6,        /* admission refused: no free slot or not enough free memory */
  DOBFS_ERR_IO = -7,          /* graph file: cannot open, read or write, or not a valid graph file */
  DOBFS_ERR_BOUNDS = -8       /* bounds-check builds only: a device index check failed (see below) */
} dobfs_status;

typedef struct dobfs_graph dobfs_graph;

/* ------------------------------------------------------------------ memory */

/* Device allocator hook. Every device buffer the library owns (graph CSR,
 * per-graph BFS workspace, build scratch) comes from `alloc` and goes back
 * through `free`. `alloc` returns NULL on failure (the call then fails with
 * DOBFS_ERR_OOM). Passing NULLs restores the default (cudaMalloc/cudaFree).
 * Process-wide; set it before creating graphs. The Python binding installs
 * PyTorch's caching allocator here. */
typedef void* (*dobfs_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*dobfs_free_fn)(void* ptr, void* stream, void* ctx);
int dobfs_set_allocator(dobfs_alloc_fn alloc, dobfs_free_fn free_fn, void* ctx);

/* Thread-local text of the last failure ("" if none). */
const char* dobfs_last_error(void);

/* ------------------------------------------------------------------ graphs */

/* Graph build flags. */
#define DOBFS_GRAPH_SYMMETRIZE 0x1u   /* add v->u for every stored u->v */
#define DOBFS_GRAPH_REINDEX 0x2u      /* degree-sorted renumbering by degree class (Sec. 3.4) */
#define DOBFS_GRAPH_DEVICE_PTRS 0x4u  /* inputs are device pointers (skip detection) */
#define DOBFS_GRAPH_VALIDATE 0x8u     /* reject input that is not symmetric */
#define DOBFS_GRAPH_OFFSETS64 0x10u   /* store int64 row offsets even if int32 would do */
#define DOBFS_GRAPH_REINDEX_EXACT 0x20u /* degree-sorted renumbering by exact degree (Sec. 3.4) */
#define DOBFS_GRAPH_CHUNKED 0x40u     /* dobfs_graph_create_rmat: build in chunks of source rows even
                                         if the one-shot key buffers would fit (same result) */

/*
 * Builds a graph from CSR arrays: row_offsets[n_vertices+1] (int32, or int64
 * if offsets_are_int64) and col_indices[n_entries] (int32). The stored graph
 * is undirected CSR with each undirected edge held as two directed edges
 * (Sec. 4, "Methodology"): self-loops and duplicate entries are dropped and
 * each row is sorted. With DOBFS_GRAPH_SYMMETRIZE the reverse of every entry
 * is added first; without it the input must already be symmetric, which
 * DOBFS_GRAPH_VALIDATE checks (DOBFS_ERR_BAD_GRAPH otherwise).
 * With DOBFS_GRAPH_REINDEX_EXACT vertices are renumbered by decreasing
 * degree (ties by increasing original ID) and every row is sorted by the new
 * IDs, which puts the highest-degree neighbour first (Sec. 3.4).
 * DOBFS_GRAPH_REINDEX renumbers by decreasing degree class instead: degrees
 * below 8 are their own class, degrees in [8, 4096) fall into four classes
 * per octave (the two bits after the leading one), degrees of 4096 or more
 * keep their exact order; ties by increasing original ID. Rows then start
 * with a neighbour of the highest class, and consecutive original IDs of a
 * class get consecutive new IDs, which keeps the translation of the results
 * back to original IDs close to sequential.
 * Row offsets are stored as int32 when the entry count fits, else int64.
 * Errors: DOBFS_ERR_INVALID (n_vertices < 1 or > 2^31-1, negative sizes,
 * NULL pointers with n_entries > 0), DOBFS_ERR_BAD_GRAPH (column or offset
 * out of range), DOBFS_ERR_OOM, DOBFS_ERR_CUDA. On success *out owns all
 * device memory of the graph; release it with dobfs_graph_destroy.
 * The build runs on `stream`; the call returns once the graph is ready.
 */
int dobfs_graph_create(const void* row_offsets, int offsets_are_int64, const int32_t* col_indices,
                       int64_t n_vertices, int64_t n_entries, uint32_t flags, void* stream,
                       dobfs_graph** out);

/*
 * Builds a graph from n_pairs undirected pairs (src[i], dst[i]) (int32 IDs in
 * [0, n_vertices)): every pair u != v is stored both ways, self-loops and
 * duplicates dropped. Flags as for dobfs_graph_create (SYMMETRIZE is implied).
 */
int dobfs_graph_create_from_pairs(const int32_t* src, const int32_t* dst, int64_t n_pairs,
                                  int64_t n_vertices, uint32_t flags, void* stream, dobfs_graph** out);

/*
 * Builds the R-MAT graph of `scale` (2^scale vertices, n_pairs undirected
 * pairs) drawn on the device by the seeded counter-based generator of
 * dobfs_inputs/gen.h, the stand-in for the Graph500 generator of Sec. 4
 * ("Workloads"): quadrant cut points t_a <= t_ab <= t_abc on a 32-bit uniform
 * draw (floor(2^32 * A), floor(2^32 * (A+B)), floor(2^32 * (A+B+C))),
 * endpoints relabelled by the seeded bijection. scale in [1, 31].
 */
int dobfs_graph_create_rmat(int scale, int64_t n_pairs, uint32_t t_a, uint32_t t_ab, uint32_t t_abc,
                            uint64_t seed, uint32_t flags, void* stream, dobfs_graph** out);

/*
 * Builds a Chung-Lu graph on n_vertices vertices from n_pairs pairs whose
 * endpoints are drawn with probability proportional to the integer weights
 * given as the inclusive cumulative table cdf[n_vertices] (host memory,
 * non-decreasing, cdf[n-1] > 0), relabelled by the seeded bijection.
 */
int dobfs_graph_create_chunglu(const uint64_t* cdf, int64_t n_vertices, int64_t n_pairs, uint64_t seed,
                               uint32_t flags, void* stream, dobfs_graph** out);

int dobfs_graph_destroy(dobfs_graph* g);

typedef struct {
  int64_t n_vertices;
  int64_t n_entries;        /* stored directed entries (2 x undirected edges) */
  int64_t n_nonisolated;    /* vertices with degree >= 1 */
  int64_t max_degree;
  int32_t offsets_int64;    /* 1 if row offsets are stored as int64 */
  int32_t reindexed;        /* 1 if DOBFS_GRAPH_REINDEX was applied */
  int64_t device_bytes;     /* graph + BFS workspace held on the device */
  float build_ms;           /* device time of the build */
} dobfs_graph_info;

int dobfs_graph_get_info(const dobfs_graph* g, dobfs_graph_info* info);

/*
 * Copies the stored CSR out in the internal vertex order: offsets_out[n+1]
 * (int64), cols_out[n_entries] (int32), new2orig_out[n] (int32; internal ID
 * -> original ID, identity when not reindexed). Any of the three may be NULL.
 * Host or device pointers.
 */
int dobfs_graph_export(const dobfs_graph* g, int64_t* offsets_out, int32_t* cols_out, int32_t* new2orig_out,
                       void* stream);

/* Degree of every vertex, indexed by original ID: deg_out[n] (int32, host or device). */
int dobfs_graph_degrees(const dobfs_graph* g, int32_t* deg_out, void* stream);

/*
 * Graph files: a built graph saved to disk and loaded again without a
 * rebuild. The file holds the stored CSR in the internal vertex order (row
 * offsets at their stored width, columns) and, for a renumbered graph, the
 * map to original IDs, after a 64-byte header with a payload checksum;
 * sections are padded to 8 bytes. Data moves through two pinned staging
 * buffers of 64 MB, so the host never holds the whole graph.
 *
 * dobfs_graph_save writes g to `path` (created or truncated) on `stream`
 * (NULL = the graph's stream), after any run still in flight on g.
 * Errors: DOBFS_ERR_INVALID (NULL argument), DOBFS_ERR_IO (the file cannot
 * be written; no partial file is left), DOBFS_ERR_OOM (staging buffers),
 * DOBFS_ERR_CUDA.
 *
 * dobfs_graph_load builds a graph from such a file. Before any BFS kernel
 * sees it, the stored CSR is checked on the device for every invariant the
 * build establishes: offsets non-decreasing from 0 to n_entries, columns in
 * range, rows strictly increasing without self-loops, and for a renumbered
 * graph degree classes non-increasing along the internal IDs and a map that
 * is a permutation. flags: 0 or DOBFS_GRAPH_VALIDATE (also check symmetry).
 * Errors: DOBFS_ERR_INVALID (NULL argument, other flags), DOBFS_ERR_IO
 * (cannot open, truncated, wrong magic or version, bad header, trailing
 * data, checksum mismatch), DOBFS_ERR_BAD_GRAPH (an invariant fails),
 * DOBFS_ERR_OOM, DOBFS_ERR_CUDA. On success *out is a graph equal to the
 * one saved (same CSR, map and results); release it with dobfs_graph_destroy.
 */
int dobfs_graph_save(const dobfs_graph* g, const char* path, void* stream);
int dobfs_graph_load(const char* path, uint32_t flags, void* stream, dobfs_graph** out);

/* ------------------------------------------------------------------ single-source runs */

/* Direction policy for a level. */
#define DOBFS_DIR_AUTO 0        /* alpha/beta heuristic on the device (default) */
#define DOBFS_DIR_TOPDOWN 1     /* every level top-down */
#define DOBFS_DIR_BOTTOMUP 2    /* every level bottom-up */
#define DOBFS_DIR_RANDOM 3      /* seeded coin per level (exercises every switch; testing) */
#define DOBFS_DIR_STATIC 4      /* the paper's policy (Sec. 3.3): the next frontier is
                                   estimated as static_pct percent of the edges out of the
                                   current one; top-down until that estimate exceeds n/beta,
                                   then bottom-up for bu_steps levels, then top-down */

/* Run flags. */
#define DOBFS_RUN_CANONICAL_PARENT 0x1u /* parent = smallest original-ID neighbour one level up */
#define DOBFS_RUN_HOST_LOOP 0x2u        /* drive levels from the host and time every kernel
                                           (diagnostics; adds one host round trip per level) */
#define DOBFS_RUN_SYNC_STATS 0x4u       /* wait for completion and fill *stats */
#define DOBFS_RUN_LEVEL_GRAPH 0x8u      /* run the level loop as the CUDA graph also for a small
                                           graph (by default a graph with at most 2^21 vertices
                                           that have edges and 2^27 stored entries runs all its
                                           levels in one cooperative kernel; same results; where
                                           the device refuses that launch, the graph uses the
                                           level graph from then on) */

typedef struct {
  int32_t direction;        /* DOBFS_DIR_* */
  int32_t alpha;            /* top-down -> bottom-up when m_f * alpha > m_u (default 14) */
  int32_t beta;             /* bottom-up -> top-down when n_f * beta < n and shrinking (default 24) */
  int32_t static_pct;       /* DOBFS_DIR_STATIC: percent of frontier out-edges (default 10) */
  int32_t bu_steps;         /* DOBFS_DIR_STATIC: bottom-up levels before returning (default 3) */
  uint32_t flags;           /* DOBFS_RUN_* */
  uint64_t schedule_seed;   /* DOBFS_DIR_RANDOM */
  void* stream;             /* cudaStream_t (NULL: the graph's creation stream) */
  int32_t td_bitmap_div;    /* a top-down level with m_f * td_bitmap_div >= n marks a next-frontier
                               bitmap and finds parents afterwards (0: never; default 2) */
  /* Degree-bin cutoffs of the step kernels (0: the path's default). They
     change only the speed, never the result. */
  int32_t td_small_max;     /* top-down rows of at most this many entries are expanded by one
                               thread, longer ones are cut into chunk records (8..256; default 16;
                               single-source runs) */
  int32_t td_chunk;         /* entries per top-down chunk record, expanded by one warp (multiple
                               of 128 in 256..8192; default 512 single-source, 1024 batched) */
  int32_t bu_scan;          /* bottom-up entries one thread scans before the rest of the row goes
                               to a warp (1..256; default 32) */
  int32_t td_split_pct;     /* mixed levels (degree-sorted graphs): a bitmap-output top-down level
                               searches the vertices of degree >= td_split_pct/100 * nnz / m_f
                               bottom-up and expands only the rest of each frontier row top-down
                               (0: off; 0..100000; default 150) */
  /* Threads per block of the step kernels (0: the default 256; else 128,
     256 or 512). Like the cutoffs they change only the speed. */
  int32_t bu_threads;       /* bottom-up search (single-source and batched runs) */
  int32_t td_threads;       /* top-down expansion (single-source and batched runs) */
  int32_t out_threads;      /* output pass (single-source runs) */
} dobfs_run_opts;

typedef struct {
  float device_ms;          /* CUDA-event time from status init to outputs written */
  int32_t levels;           /* number of BFS levels (max level + 1) */
  int32_t td_levels;        /* levels expanded top-down */
  int32_t bu_levels;        /* levels expanded bottom-up */
  int64_t reached;          /* vertices reached */
  int64_t teps_edges;       /* undirected edges in the root's component */
  int64_t edges_examined;   /* adjacency entries read by the level kernels */
  int64_t alg_bytes;        /* algorithmic DRAM bytes of the run: the sum over levels of
                               top-down (queue output): 20 n_f + 4 m_f + 12 n_new
                                 (+ 4 n_f after a bitmap -> queue conversion);
                               bottom-up: 8 n_scanned + 4 e_examined + 8 n_new
                                 (+ 4 n_f after a queue -> bitmap conversion);
                               top-down with bitmap output and mixed levels:
                                 24 n_f + 4 e_examined + 8 n_scanned + 12 n_new;
                               plus the output pass: 8 n (level and parent written)
                                 + 4 n (map read, renumbered graphs) + 8 reached
                                 ((level, parent) gathered). Frontier and visited
                               bitmaps are counted as L2 traffic, not DRAM. */
} dobfs_run_stats;

/* Fills *opts with the defaults. */
int dobfs_run_opts_init(dobfs_run_opts* opts);

/*
 * One BFS from `root` (original ID). level_out[n] and parent_out[n] (int32,
 * indexed by original ID; parent_out may be NULL) receive the BFS level and
 * a BFS parent (any frontier neighbour one level up, or the canonical one
 * with DOBFS_RUN_CANONICAL_PARENT). Host or device pointers. Asynchronous on
 * the run's stream unless stats are requested (DOBFS_RUN_SYNC_STATS or a
 * non-NULL stats) or the outputs are host memory.
 * Errors: DOBFS_ERR_INVALID (NULL graph/level_out, root out of range, bad
 * opts), DOBFS_ERR_CUDA, DOBFS_ERR_OOM (host-output staging).
 */
int dobfs_run(dobfs_graph* g, int32_t root, int32_t* level_out, int32_t* parent_out,
              const dobfs_run_opts* opts, dobfs_run_stats* stats);

/*
 * Waits at most timeout_ms milliseconds (< 0: no limit; 0: only test) for
 * the work the library has queued for g: its last run or batch, on whatever
 * stream it ran, with everything queued before it on that stream. Runs and
 * batches with device outputs return once launched; this bounds the wait for
 * them. Returns DOBFS_OK once that work is done (or if none was queued),
 * DOBFS_ERR_TIMEOUT if it is still running at the limit (nothing is
 * cancelled: it completes later, and a later wait returns DOBFS_OK),
 * DOBFS_ERR_CUDA if it failed, DOBFS_ERR_INVALID for a NULL graph. The
 * graph must not be destroyed during the wait. No kernel of the library
 * waits for another kernel: the level loop is a CUDA graph whose conditional
 * nodes end it on the device, or, for a small graph, one cooperative kernel
 * whose blocks (all resident at once) meet at grid barriers, each wait there
 * bounded by 2 s (a wait that runs out fails the run with DOBFS_ERR_CUDA
 * when its stats are read).
 */
int dobfs_graph_wait(dobfs_graph* g, int32_t timeout_ms);

/*
 * Batched BFS from n_roots roots (original IDs) with the bit-parallel
 * multi-source traversal: roots are the lanes of traversals in which every
 * vertex carries lane masks (lanes that reached it, lanes for which it is in
 * the frontier): up to 64 roots run as one 64-lane traversal, more in
 * traversals of 128 lanes (two 64-bit mask words per vertex; a wide
 * bottom-up level scans whole rows whatever the lane count, so 128 lanes
 * cost about what 64 do); each level runs top-down or
 * bottom-up (Algorithm 1) for all lanes at once, the direction picked by the
 * alpha/beta rule on the union of the lanes' frontiers. level_out[n_roots][n]
 * (int32, row r for roots[r], original IDs) receives the levels, identical
 * to n_roots separate dobfs_run calls. Levels only: parent_out must be NULL.
 * n_roots = 0 does nothing (roots and level_out may then be NULL).
 * roots and level_out may be host or device memory. A lane runs at most 65535
 * levels. opts: direction auto, top-down, bottom-up or random; alpha, beta,
 * td_chunk, bu_scan, schedule_seed, stream; with opts NULL, the defaults of
 * dobfs_run_opts_init except alpha = DOBFS_BATCH_ALPHA (the union frontier of
 * 64 lanes reaches a bottom-up size sooner than one lane's). stats
 * (nullable): device_ms, levels (deepest group), edges_examined, and
 * alg_bytes: per step of a lane group of W mask words (64 W lanes), 16 W
 * bytes per active vertex (its seen and next masks; a top-down step's
 * frontier vertices, a bottom-up step's searched vertices) + (8 W + 4) per
 * examined entry (the neighbour's frontier mask and the column), plus 4
 * bytes per (vertex, root) level written by the flush.
 * Asynchronous on the batch's stream when level_out is device memory and
 * stats is NULL (device roots are first read back with a synchronous copy);
 * otherwise the call returns when the levels are written.
 */
#define DOBFS_BATCH_ALPHA 4
int dobfs_run_batch(dobfs_graph* g, const int32_t* roots, int32_t n_roots, int32_t* level_out, int32_t* parent_out,
                    const dobfs_run_opts* opts, dobfs_run_stats* stats);

/* ------------------------------------------------------------------ serving */

/*
 * A query server over resident graphs with continuous batching: queries
 * (graph, root) are admitted as they arrive into free lanes of 128-lane
 * (or, with lane_words = 1, 64-lane) bit-parallel traversals already running
 * on that graph (lanes join and
 * leave at level boundaries), each graph's lane groups run on their own
 * CUDA streams so work overlaps on the device, and a scheduler thread owned
 * by the server drives the levels. Each level is a step of Algorithm 1 for
 * all lanes of a group, top-down or bottom-up by the alpha/beta rule on the
 * union of the lanes' frontiers. A query's result is the level array of a
 * lone BFS from its root, whatever else is in flight. Levels only.
 *
 * Lanes of a group form cohorts: an idle group starts one with the queries
 * waiting for its graph, and later arrivals join it only within join_window
 * levels of its start (while the levels are light), so the wide middle
 * levels of its lanes coincide; other arrivals go to the graph's other
 * groups. Under light load (a graph with at most ss_max waiting queries) a
 * query instead runs as a single-source BFS on that graph's own stream, which
 * answers one query faster than a lane group does. The server expects to be
 * the only user of its graphs while it runs. Admission: a query takes a free lane of its graph and, if its output is
 * host memory, a device staging buffer of n int32 counted against
 * max_device_bytes; queries wait (in arrival order per graph) until both are
 * available. More lane groups (up to max_groups_per_graph) are created while
 * queries wait and the budget allows. A group of W mask words (64 W lanes)
 * holds 8 W bytes per vertex for each of its 3 + 16 masks (lanes seen,
 * current and next frontier, and 16 bit planes of the discovery level):
 * 152 W bytes per vertex, i.e. 152 for 64 lanes and 304 for the default 128,
 * plus 4 bytes per vertex for deferred rows and 8-byte top-down records (one
 * per vertex with an edge, and one per 256 stored entries).
 */
typedef struct dobfs_server dobfs_server;

typedef struct {
  int64_t max_device_bytes;     /* device-memory budget for lane groups and staging (0: 90% of free memory) */
  int32_t groups_per_graph;     /* lane groups created per graph up front (default 1) */
  int32_t max_groups_per_graph; /* upper bound on groups per graph (default 1: one full cohort at a time
                                   beats two half-full ones, since a wide step costs the same either way) */
  int32_t alpha, beta;          /* direction rule of the lane groups (defaults DOBFS_BATCH_ALPHA, 24);
                                   the single-source path uses dobfs_run_opts_init's */
  int32_t direction;            /* DOBFS_DIR_AUTO / TOPDOWN / BOTTOMUP / RANDOM */
  int32_t admit_div;            /* a busy group admits new queries only at levels whose union frontier
                                   n_f satisfies n_f * admit_div < n (0: at every level; default 64) */
  int32_t join_window;          /* ... and only within this many levels of its cohort's start; an idle
                                   group always admits (default 1; large values: join at any light level) */
  int32_t flush_delay;          /* finished lanes of a group are written out together when no lane is
                                   left running, or once the oldest has waited this many levels
                                   (default 3; 0: at once) */
  int32_t gather_us;            /* an idle group starts a cohort when a full group of queries (64 *
                                   lane_words) waits or the oldest has waited this long (default
                                   2000 us; 0: at once) */
  int32_t ss_max;               /* while at most this many queries of a graph wait, they run as single-
                                   source BFS (dobfs_run) on the graph's own stream instead (device
                                   outputs only; default 2; 0: never) */
  int32_t ss_backlog;           /* ... as long as fewer than this many are already queued there (default 4) */
  int32_t lane_words;           /* lanes per group: 64 * lane_words, 1 or 2 (default 2: a wide bottom-up
                                   step scans whole rows anyway, so 128 lanes cost about what 64 do) */
} dobfs_serve_opts;

typedef struct {
  int32_t status;      /* DOBFS_OK, or the error that failed the query */
  int32_t levels;      /* levels of the query's BFS (max level + 1) */
  int64_t submit_ns;   /* CLOCK_MONOTONIC time of dobfs_serve_submit */
  int64_t admit_ns;    /* when the query took a lane */
  int64_t done_ns;     /* when its output was complete and visible to poll */
  int64_t latency_ns;  /* done_ns - submit_ns */
} dobfs_query_result;

typedef struct {
  int64_t iterations;      /* scheduler passes that did work */
  int64_t completed;       /* queries finished */
  int64_t in_flight;       /* submitted and not yet polled */
  int64_t groups_created;  /* lane groups added beyond the initial ones */
  int64_t reserved_bytes;  /* device memory held against the budget */
  int64_t budget_bytes;
  int64_t cohorts;         /* traversals started by an idle lane group */
  int64_t lanes_admitted;  /* queries that took a lane (lanes_admitted / cohorts: mean cohort size) */
  int64_t group_steps;     /* levels stepped by lane groups */
  int64_t single_source;   /* queries served by the single-source path */
} dobfs_serve_stats;

int dobfs_serve_opts_init(dobfs_serve_opts* opts);
/* Starts the server (and its scheduler thread) on the current device. */
int dobfs_serve_create(const dobfs_serve_opts* opts, dobfs_server** out);
/* Adds a resident graph (it must outlive the server); *gid identifies it in submissions.
 * DOBFS_ERR_BUSY if the budget cannot hold its initial lane groups. */
int dobfs_serve_add_graph(dobfs_server* s, dobfs_graph* g, int32_t* gid);
/* Queues the query (gid, root); level_out[n] (host or device) must stay valid until poll
 * returns DOBFS_OK. parent_out must be NULL. Never blocks on the GPU. */
int dobfs_serve_submit(dobfs_server* s, int32_t gid, int32_t root, int32_t* level_out, int32_t* parent_out,
                       uint64_t* ticket);
/* DOBFS_PENDING while the query runs; DOBFS_OK (result filled, ticket retired) once
 * level_out is complete; an error status if the query failed (ticket retired). */
int dobfs_serve_poll(dobfs_server* s, uint64_t ticket, dobfs_query_result* result);
/* Retires up to max_results finished queries in completion order without naming them:
 * tickets[i] and results[i] for i < *n_out (for load generators that track many tickets). */
int dobfs_serve_collect(dobfs_server* s, uint64_t* tickets, dobfs_query_result* results, int32_t max_results,
                        int32_t* n_out);
int dobfs_serve_get_stats(dobfs_server* s, dobfs_serve_stats* stats);
/* Stops the scheduler and frees the server (unpolled queries are dropped). */
int dobfs_serve_destroy(dobfs_server* s);

/* Per-level record of the last run on a graph (ready after that run completed). */
typedef struct {
  int32_t level;            /* level L being expanded (frontier = vertices at level L) */
  int32_t direction;        /* 0 top-down, 1 bottom-up, 2 mixed (bottom-up for the high-degree
                               vertices, top-down for the rest; see td_split_pct) */
  int64_t n_frontier;       /* n_f: vertices at level L */
  int64_t m_frontier;       /* m_f: sum of their degrees */
  int64_t m_unvisited;      /* m_u: sum of degrees of unvisited vertices before the step */
  int64_t n_next;           /* vertices discovered (level L+1) */
  int64_t edges_examined;
  int64_t vertices_scanned; /* bottom-up: unvisited vertices scanned */
  int64_t alg_bytes;
  float ms;                 /* host-loop runs only: device time of the level's kernels, else 0 */
  float ms_main;            /* host-loop runs only: time of the main expand kernel */
} dobfs_level_trace;

/* Copies up to max_levels records of the last run; *n_out = records written. */
int dobfs_last_trace(const dobfs_graph* g, dobfs_level_trace* out, int32_t max_levels, int32_t* n_out);

/* ------------------------------------------------------------------ allocation-free runs */

/*
 * The paper has no counterpart of this entry point; it exists for callers
 * that cannot allocate device memory when they need a BFS: code working in
 * a memory budget reserved up front, allocation-free real-time or serving
 * paths, or plugins inside a framework that owns every device allocation.
 * dobfs_run needs a graph from dobfs_graph_create, which allocates; this
 * call allocates nothing (no cudaMalloc, no cudaFree, no allocating library
 * routine).
 *
 * BFS from `root` on the caller's CSR: row_offsets[n_vertices+1] (int32) and
 * col_indices[row_offsets[n_vertices]] (int32), both device pointers, the
 * graph undirected (every edge stored both ways). Every row_offsets entry
 * must lie in [0, row_offsets[n_vertices]] and be non-decreasing, and every
 * col_indices entry in [0, n_vertices): the normal build reads and writes
 * through these values unchecked (a column at or past n_vertices writes
 * past level_out and the working memory); the bounds-check build
 * libdobfs_bc.so checks each of them on the device and returns
 * DOBFS_ERR_BOUNDS instead. level_out[n_vertices] and
 * parent_out[n_vertices] (device pointers; parent_out may be NULL) receive
 * the level (-1 if unreached) and a BFS parent (parent[root] = root).
 *
 * Working memory: one static device array of about 8.4 MB, sized for at
 * most DOBFS_STATIC_MAX_VERTICES vertices, held by every GPU that loads the
 * library until the process exits. n_vertices above that maximum (or below
 * 1), a root out of range or a NULL pointer give DOBFS_ERR_INVALID before
 * any GPU work.
 *
 * Every call looks up the array's device address on the current device with
 * cudaGetSymbolAddress (a lookup, not an allocation), so a call made after
 * cudaDeviceReset uses the new context's array. The call is synchronous:
 * it reads two row offsets and, after every level, a few counters back to
 * the host and synchronises `stream` each time, and returns when the BFS is
 * done. It therefore cannot be called on a stream that is being captured
 * into a CUDA graph. Every call on a device shares the array and clears
 * what must start at zero. The library serialises calls, so calls through
 * this entry point do not overlap; GPU work that overlapped with a call
 * (for instance a second copy of this library in the process using its own
 * lock) would race on the array. Levels are chosen by the alpha/beta rule
 * with the defaults of dobfs_run_opts_init.
 */
#define DOBFS_STATIC_MAX_VERTICES (1 << 20)
int dobfs_run_static(const int32_t* row_offsets, const int32_t* col_indices, int32_t n_vertices, int32_t root,
                     int32_t* level_out, int32_t* parent_out, void* stream);

/* ------------------------------------------------------------------ bounds-check builds */

/*
 * libdobfs_bc.so is this library compiled with -DDOBFS_BOUNDS_CHECK. Every
 * index its kernels read from memory (a vertex ID from a column, queue,
 * record or map; a row's offsets; a write position taken from a counter) is
 * checked on the device before use. A failing check records where it
 * failed and substitutes a safe value, so the access stays in bounds; the
 * call then returns DOBFS_ERR_BOUNDS with the place named in
 * dobfs_last_error() (a server fails its queries with that status). Every
 * device buffer is over-allocated by 64 KB, room for 1024 vertex IDs past
 * n in any per-vertex array. The normal build compiles the checks away.
 *
 * dobfs_debug_set_column (bounds-check builds only; DOBFS_ERR_INVALID
 * otherwise) overwrites stored entry `pos` (internal order, [0, n_entries))
 * with `value`, which must lie in [0, n + 1024): a corrupted graph for
 * testing the checks. The graph's first-neighbour table is refreshed.
 */
int dobfs_debug_set_column(dobfs_graph* g, int64_t pos, int32_t value);

/*
 * Self-test of the grid barrier that the fused level loop of small graphs
 * uses between phases (all builds). One cooperative launch of `blocks`
 * blocks (1 up to the resident capacity) runs `rounds` barriers (0..2^20);
 * before each, every block adds one to a counter, after it one block
 * checks that the counter holds every block's additions. With missing = 1
 * the barrier waits for one block more than was launched, so every wait
 * runs out after its 2 s bound and the launch ends without a fault. Out:
 * *rounds_passed (rounds whose barrier completed), *short_counts (rounds
 * that saw a counter short of a block's addition: 0 for a correct
 * barrier), *timed_out (1 if a wait ran out). Synchronous, on the legacy
 * default stream; allocates 32 bytes through the allocator hook.
 * Errors: DOBFS_ERR_INVALID (NULL outputs, arguments out of range),
 * DOBFS_ERR_CUDA, DOBFS_ERR_OOM.
 */
int dobfs_debug_grid_barrier(int32_t blocks, int32_t rounds, int32_t missing, int32_t* rounds_passed,
                             int32_t* short_counts, int32_t* timed_out);

/*
 * Measurement aid for the rooflines of the BFS steps, whose memory accesses
 * are mostly scattered reads and writes of 4 to 16 bytes (all builds).
 * Allocates array_bytes of device memory (a power of two, at least 1 MB)
 * through the allocator hook, then times one launch that makes at least
 * `accesses` accesses of `width` bytes (4, 8 or 16; reads, or writes with
 * write = 1) at positions drawn by a hash, eight in flight per thread, over
 * every SM. Out: *ms_out (CUDA-event time of the launch, after one untimed
 * launch) and *made_out (accesses made: the request rounded up to whole
 * rounds of the grid). Synchronous, on the legacy default stream.
 * Errors: DOBFS_ERR_INVALID (NULL outputs, arguments out of range),
 * DOBFS_ERR_OOM, DOBFS_ERR_CUDA.
 */
int dobfs_debug_random_access(int64_t array_bytes, int64_t accesses, int32_t width, int32_t write,
                              float* ms_out, int64_t* made_out);

#ifdef __cplusplus
}
#endif

#endif /* DOBFS_H */
