/*
 * CPU oracle for direction-optimized BFS — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use
 * this file. It shares no code with the CUDA library; the only code both
 * include is the seeded input generator (dobfs_inputs/gen.h).
 *
 * What the method computes, and what this oracle writes out plainly:
 * direction-optimized BFS (Sec. 2.2; Algorithm 1) produces the same next
 * frontier whether a level is expanded top-down or bottom-up, so its level
 * array is the plain BFS distance from the root. The oracle is therefore a
 * serial FIFO-queue BFS over the undirected graph stored as CSR with each
 * undirected edge held as two directed edges (Sec. 4, "Methodology").
 * Parents follow the Graph500 requirement of a BFS parent tree (Sec. 4,
 * "Methodology"); since Algorithm 1 admits any frontier neighbour as parent,
 * the oracle's parent is the canonical one: the smallest-ID neighbour one
 * level up.
 *
 * Conventions (the paper states none): unreached vertices have level -1 and
 * parent -1; parent[root] = root.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "../dobfs_inputs/gen.h"

static int cmp_i32(const void* a, const void* b) {
  const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Sort each row, drop duplicate entries, compact in place. off[] is
 * rewritten; returns the new number of stored entries. */
static int64_t sort_dedup_rows(int64_t n, int64_t* off, int32_t* cols) {
  int64_t w = 0;
  int64_t row_start = off[0];
  for (int64_t u = 0; u < n; ++u) {
    const int64_t s = row_start, e = off[u + 1];
    row_start = e;
    qsort(cols + s, (size_t)(e - s), sizeof(int32_t), cmp_i32);
    off[u] = w;
    for (int64_t j = s; j < e; ++j) {
      if (j > s && cols[j] == cols[j - 1]) continue;
      cols[w++] = cols[j];
    }
  }
  off[n] = w;
  return w;
}

/*
 * CSR of the undirected graph given by m pairs (src[i], dst[i]): every pair
 * u != v is stored as u->v and v->u; self-loops and duplicates are dropped;
 * each row is sorted ascending. Textbook counting placement: count entries
 * per row, prefix-sum, scatter, then sort and de-duplicate each row.
 * off must hold n+1 entries, cols 2*m. Returns the number of stored entries
 * (directed edges), or -1 on an out-of-range endpoint.
 */
int64_t oracle_csr_from_pairs(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                              int64_t* off, int32_t* cols) {
  memset(off, 0, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t i = 0; i < m; ++i) {
    const int32_t u = src[i], v = dst[i];
    if (u < 0 || v < 0 || u >= n || v >= n) return -1;
    if (u == v) continue;
    off[u + 1]++;
    off[v + 1]++;
  }
  for (int64_t u = 0; u < n; ++u) off[u + 1] += off[u];
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  memcpy(pos, off, sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < m; ++i) {
    const int32_t u = src[i], v = dst[i];
    if (u == v) continue;
    cols[pos[u]++] = v;
    cols[pos[v]++] = u;
  }
  free(pos);
  return sort_dedup_rows(n, off, cols);
}

/* Same CSR, with the pairs regenerated from the R-MAT stream of gen.h
 * instead of being held in memory (two passes over the stream). */
int64_t oracle_csr_from_rmat(int scale, int64_t m, uint32_t t_a, uint32_t t_ab, uint32_t t_abc,
                             uint64_t seed, int64_t* off, int32_t* cols) {
  const int64_t n = (int64_t)1 << scale;
  const uint64_t kp = gen_key_pairs(seed), kq = gen_key_perm(seed);
  memset(off, 0, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t i = 0; i < m; ++i) {
    uint32_t u, v;
    gen_rmat_pair((uint64_t)i, scale, t_a, t_ab, t_abc, kp, kq, &u, &v);
    if (u == v) continue;
    off[u + 1]++;
    off[v + 1]++;
  }
  for (int64_t u = 0; u < n; ++u) off[u + 1] += off[u];
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  memcpy(pos, off, sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < m; ++i) {
    uint32_t u, v;
    gen_rmat_pair((uint64_t)i, scale, t_a, t_ab, t_abc, kp, kq, &u, &v);
    if (u == v) continue;
    cols[pos[u]++] = (int32_t)v;
    cols[pos[v]++] = (int32_t)u;
  }
  free(pos);
  return sort_dedup_rows(n, off, cols);
}

/* Source of the undirected pairs of a streamed graph: regenerated R-MAT
 * pairs (gen.h), or pairs held in two arrays. */
typedef struct {
  int kind; /* 0: R-MAT stream, 1: arrays */
  int scale;
  uint32_t t_a, t_ab, t_abc;
  uint64_t kp, kq;
  const int32_t* src;
  const int32_t* dst;
} pair_source;

static inline void get_pair(const pair_source* ps, int64_t i, uint32_t* u, uint32_t* v) {
  if (ps->kind == 0) {
    gen_rmat_pair((uint64_t)i, ps->scale, ps->t_a, ps->t_ab, ps->t_abc, ps->kp, ps->kq, u, v);
  } else {
    *u = (uint32_t)ps->src[i];
    *v = (uint32_t)ps->dst[i];
  }
}

/*
 * The CSR of oracle_csr_from_rmat / oracle_csr_from_pairs built by n_threads
 * threads, for graphs of billions of entries (R-MAT scale 28: 8.6 G entries
 * before de-duplication). Same counting placement, spread over threads: the
 * pair stream is split into ranges, each thread counts its pairs' endpoints
 * into the row counts with atomic increments; after the prefix sum each
 * thread places its pairs at atomically advanced row cursors (so the order
 * inside a row differs from the serial placement, which the row sort
 * removes); rows are then sorted and de-duplicated in parallel, and finally
 * moved down over the removed duplicates in row order. The result equals
 * the serial builders'.
 */
static int64_t csr_par_core(const pair_source* ps, int64_t n, int64_t m, int64_t* off, int32_t* cols, int nt) {
  (void)nt;
  memset(off, 0, sizeof(int64_t) * (size_t)(n + 1));
#pragma omp parallel for schedule(static, 1 << 16) num_threads(nt)
  for (int64_t i = 0; i < m; ++i) {
    uint32_t u, v;
    get_pair(ps, i, &u, &v);
    if (u == v) continue;
    __atomic_fetch_add(&off[u + 1], 1, __ATOMIC_RELAXED);
    __atomic_fetch_add(&off[v + 1], 1, __ATOMIC_RELAXED);
  }
  for (int64_t u = 0; u < n; ++u) off[u + 1] += off[u];
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  memcpy(pos, off, sizeof(int64_t) * (size_t)n);
#pragma omp parallel for schedule(static, 1 << 16) num_threads(nt)
  for (int64_t i = 0; i < m; ++i) {
    uint32_t u, v;
    get_pair(ps, i, &u, &v);
    if (u == v) continue;
    cols[__atomic_fetch_add(&pos[u], 1, __ATOMIC_RELAXED)] = (int32_t)v;
    cols[__atomic_fetch_add(&pos[v], 1, __ATOMIC_RELAXED)] = (int32_t)u;
  }
  /* sort each row and drop its duplicates in place; pos[u] = kept length */
#pragma omp parallel for schedule(dynamic, 4096) num_threads(nt)
  for (int64_t u = 0; u < n; ++u) {
    const int64_t s = off[u], e = off[u + 1];
    qsort(cols + s, (size_t)(e - s), sizeof(int32_t), cmp_i32);
    int64_t w = s;
    for (int64_t j = s; j < e; ++j) {
      if (j > s && cols[j] == cols[j - 1]) continue;
      cols[w++] = cols[j];
    }
    pos[u] = w - s;
  }
  int64_t w = 0;
  for (int64_t u = 0; u < n; ++u) {
    const int64_t s = off[u], len = pos[u];
    if (w != s) memmove(cols + w, cols + s, sizeof(int32_t) * (size_t)len);
    off[u] = w;
    w += len;
  }
  off[n] = w;
  free(pos);
  return w;
}

int64_t oracle_csr_from_rmat_par(int scale, int64_t m, uint32_t t_a, uint32_t t_ab, uint32_t t_abc,
                                 uint64_t seed, int64_t* off, int32_t* cols, int32_t n_threads) {
  const pair_source ps = {0, scale, t_a, t_ab, t_abc, gen_key_pairs(seed), gen_key_perm(seed), NULL, NULL};
  return csr_par_core(&ps, (int64_t)1 << scale, m, off, cols, n_threads > 0 ? n_threads : 1);
}

/* Returns -1 on an out-of-range endpoint, like oracle_csr_from_pairs. */
int64_t oracle_csr_from_pairs_par(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int64_t* off,
                                  int32_t* cols, int32_t n_threads) {
  const int nt = n_threads > 0 ? n_threads : 1;
  int64_t bad = 0;
#pragma omp parallel for reduction(+ : bad) num_threads(nt)
  for (int64_t i = 0; i < m; ++i) bad += (src[i] < 0 || dst[i] < 0 || src[i] >= n || dst[i] >= n) ? 1 : 0;
  if (bad) return -1;
  const pair_source ps = {1, 0, 0, 0, 0, 0, 0, src, dst};
  return csr_par_core(&ps, n, m, off, cols, nt);
}

/*
 * Serial FIFO-queue BFS from `root` (plain definition of the BFS level).
 * level[v] = hop distance from root, -1 if unreachable. If parent is not
 * NULL it receives the canonical parent: for v != root reached,
 * min{u in N(v) : level[u] = level[v] - 1}; parent[root] = root; -1 for
 * unreached vertices. Returns the number of levels (max level + 1).
 */
int32_t oracle_bfs(int64_t n, const int64_t* off, const int32_t* cols, int32_t root, int32_t* level,
                   int32_t* parent) {
  for (int64_t v = 0; v < n; ++v) level[v] = -1;
  if (root < 0 || root >= n) return 0;
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t head = 0, tail = 0;
  level[root] = 0;
  queue[tail++] = root;
  int32_t maxlev = 0;
  while (head < tail) {
    const int32_t u = queue[head++];
    for (int64_t j = off[u]; j < off[u + 1]; ++j) {
      const int32_t v = cols[j];
      if (level[v] == -1) {
        level[v] = level[u] + 1;
        if (level[v] > maxlev) maxlev = level[v];
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  if (parent) {
    for (int64_t v = 0; v < n; ++v) {
      parent[v] = -1;
      if (level[v] <= 0) continue;
      for (int64_t j = off[v]; j < off[v + 1]; ++j) {
        const int32_t u = cols[j];
        if (level[u] == level[v] - 1 && (parent[v] == -1 || u < parent[v])) parent[v] = u;
      }
    }
    parent[root] = root;
  }
  return maxlev + 1;
}

/*
 * The FIFO-queue BFS of oracle_bfs, stopped once it has read max_entries
 * adjacency entries (a bounded sample of one BFS on a graph too large to
 * traverse in full on one core in the time allowed). Levels are assigned
 * when a vertex is first reached, so every level written equals the full
 * BFS level; vertices not reached by then keep -1. Returns the number of
 * entries read: every entry of every row started, so it may exceed
 * max_entries by less than one row. With max_entries >= the stored entries
 * the result is oracle_bfs's level array.
 */
int64_t oracle_bfs_partial(int64_t n, const int64_t* off, const int32_t* cols, int32_t root, int32_t* level,
                           int64_t max_entries) {
  for (int64_t v = 0; v < n; ++v) level[v] = -1;
  if (root < 0 || root >= n) return 0;
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t head = 0, tail = 0, read = 0;
  level[root] = 0;
  queue[tail++] = root;
  while (head < tail && read < max_entries) {
    const int32_t u = queue[head++];
    for (int64_t j = off[u]; j < off[u + 1]; ++j) {
      const int32_t v = cols[j];
      if (level[v] == -1) {
        level[v] = level[u] + 1;
        queue[tail++] = v;
      }
    }
    read += off[u + 1] - off[u];
  }
  free(queue);
  return read;
}

/* oracle_bfs for several roots; root r writes level[r*n ..], parent[r*n ..]. */
void oracle_bfs_many(int64_t n, const int64_t* off, const int32_t* cols, int32_t n_roots,
                     const int32_t* roots, int32_t* level, int32_t* parent, int32_t n_threads) {
  (void)n_threads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int32_t r = 0; r < n_roots; ++r)
    oracle_bfs(n, off, cols, roots[r], level + (int64_t)r * n, parent ? parent + (int64_t)r * n : NULL);
}

static int has_edge(const int64_t* off, const int32_t* cols, int32_t u, int32_t v) {
  int64_t lo = off[u], hi = off[u + 1];
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (cols[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo < off[u + 1] && cols[lo] == v;
}

static int32_t uf_find(int32_t* p, int32_t x) {
  while (p[x] != x) {
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

/* Connected components by union-find over all stored edges; comp[v] = the
 * smallest vertex ID of v's component. */
void oracle_components(int64_t n, const int64_t* off, const int32_t* cols, int32_t* comp) {
  for (int64_t v = 0; v < n; ++v) comp[v] = (int32_t)v;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t j = off[u]; j < off[u + 1]; ++j) {
      const int32_t a = uf_find(comp, (int32_t)u), b = uf_find(comp, cols[j]);
      if (a < b) comp[b] = a; else if (b < a) comp[a] = b;
    }
  for (int64_t v = 0; v < n; ++v) comp[v] = uf_find(comp, (int32_t)v);
}

/*
 * Checks a (level, parent) pair claimed to be a BFS from `root` against the
 * BFS invariants. Returns 0 if all hold, else the number of the first
 * violated rule, with the offending vertex in *bad:
 *  1  level[root] != 0
 *  2  parent[root] != root (skipped when parent is NULL)
 *  3  an edge joins two reached vertices whose levels differ by more than 1
 *  4  an edge joins a reached and an unreached vertex
 *  5  a reached v != root whose parent is not a neighbour
 *  6  a reached v != root whose parent is not exactly one level up
 *  7  an unreached vertex with level != -1 or parent != -1
 *  8  reached set differs from the root's connected component
 * 10  a reached v != root with no neighbour exactly one level up
 * Rules 1, 3, 4 and 10 together imply level = BFS distance: following
 * neighbours one level up from v reaches the root in level[v] hops, and no
 * path can be shorter since levels grow by at most one per edge.
 */
int32_t oracle_check_bfs(int64_t n, const int64_t* off, const int32_t* cols, int32_t root,
                         const int32_t* level, const int32_t* parent, int64_t* bad) {
  *bad = root;
  if (root < 0 || root >= n || level[root] != 0) return 1;
  if (parent && parent[root] != root) return 2;
  for (int64_t u = 0; u < n; ++u) {
    *bad = u;
    if (level[u] < -1) return 7;
    if (level[u] == -1) {
      if (parent && parent[u] != -1) return 7;
      continue;
    }
    for (int64_t j = off[u]; j < off[u + 1]; ++j) {
      const int32_t v = cols[j];
      if (level[v] == -1) return 4;
      if (level[v] - level[u] > 1 || level[u] - level[v] > 1) return 3;
    }
    if (u == root) continue;
    int up = 0;
    for (int64_t j = off[u]; j < off[u + 1] && !up; ++j) up = (level[cols[j]] == level[u] - 1);
    if (!up) return 10;
    if (parent) {
      const int32_t p = parent[u];
      if (p < 0 || p >= n || !has_edge(off, cols, (int32_t)u, p)) return 5;
      if (level[p] != level[u] - 1) return 6;
    }
  }
  int32_t* comp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  oracle_components(n, off, cols, comp);
  int32_t rc = 0;
  for (int64_t v = 0; v < n; ++v)
    if ((comp[v] == comp[root]) != (level[v] >= 0)) {
      *bad = v;
      rc = 8;
      break;
    }
  free(comp);
  return rc;
}

/* Undirected edges in the traversed component: (sum of degrees of reached
 * vertices) / 2, the TEPS numerator of Sec. 4 "Methodology". */
int64_t oracle_teps_edges(int64_t n, const int64_t* off, const int32_t* level) {
  int64_t s = 0;
  for (int64_t v = 0; v < n; ++v)
    if (level[v] >= 0) s += off[v + 1] - off[v];
  return s / 2;
}

static void note_violation(int32_t* rule_out, int64_t* bad_out, int32_t rule, int64_t where) {
#pragma omp critical
  {
    if (*rule_out == 0 || where < *bad_out) {
      *rule_out = rule;
      *bad_out = where;
    }
  }
}

static void atomic_min_i32(int32_t* p, int32_t x) {
  int32_t cur = __atomic_load_n(p, __ATOMIC_RELAXED);
  while ((cur == -1 || x < cur) && !__atomic_compare_exchange_n(p, &cur, x, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
  }
}

/* The rules checked per vertex after the pass over the pairs (see below):
 * 7, 10, 5, 9, 6 for vertex v of the root whose entries start at base (entry
 * of v at ov = base + v*sv); 0 if all hold. */
static int32_t vertex_rule(int64_t ov, int64_t v, int32_t root, int64_t n, const int32_t* level,
                           const int32_t* parent, const uint8_t* up, const uint8_t* confirmed, int64_t base,
                           int64_t sv) {
  const int32_t lvv = level[ov];
  if (lvv < -1) return 7;
  if (lvv == -1) return (parent && parent[ov] != -1) ? 7 : 0;
  if (v == root) return 0;
  if (!up[ov]) return 10;
  if (!parent) return 0;
  const int32_t p = parent[ov];
  if (p < 0 || p >= n) return 5;
  if (!confirmed[ov]) return 9;
  if (level[base + (int64_t)p * sv] != lvv - 1) return 6;
  return 0;
}

/*
 * Streaming check of R BFS results (roots[r], level[(r, v)], parent[(r, v)])
 * on a graph given only by its pair stream, without building a CSR. Entry
 * (r, v) of every per-root array sits at r*n + v (root-major) or, with
 * vertex_major, at v*R + r, so that a pair's levels for all roots are read
 * together (the same check; the layout only changes the memory traffic). For
 * every pair u != v (stored both ways in the graph) the edge rules 3 and 4
 * of oracle_check_bfs are checked; a pair also confirms parent[v] == u (or
 * parent[u] == v) as an edge and marks a neighbour one level up. After the
 * pass every reached v != root must have a neighbour one level up (rule 10)
 * and a confirmed parent one level up, and canon[(r, v)] receives
 * min{u in N(v) : level[u] = level[v] - 1} (canon may be NULL). has_nbr (may
 * be NULL) receives 1 for every vertex with at least one neighbour.
 * rc[r] receives 0 or the rule number as above, with bad[r] the vertex;
 * rule 9 = the parent is not a neighbour. Rule 8 needs no union-find here:
 * rule 4 makes the reached set closed under edges and rule 10 connects every
 * reached vertex to the root. Returns the number of failed roots.
 */
static int32_t check_stream_core(const pair_source* ps, int64_t n, int64_t m, int32_t R, const int32_t* roots,
                                 const int32_t* level, const int32_t* parent, int32_t* canon, uint8_t* has_nbr,
                                 int32_t n_threads, int32_t* rc, int64_t* bad, int vertex_major) {
  const int64_t sr = vertex_major ? 1 : n, sv = vertex_major ? R : 1;  /* (r, v) -> r*sr + v*sv */
  uint8_t* confirmed = (uint8_t*)calloc((size_t)(n * R), 1);
  uint8_t* up = (uint8_t*)calloc((size_t)(n * R), 1);
  if (canon)
    for (int64_t i = 0; i < n * R; ++i) canon[i] = -1;
  if (has_nbr) memset(has_nbr, 0, (size_t)n);
  for (int32_t r = 0; r < R; ++r) {
    const int32_t root = roots[r];
    rc[r] = 0;
    bad[r] = root;
    if (root < 0 || root >= n || level[r * sr + root * sv] != 0) rc[r] = 1;
    else if (parent && parent[r * sr + root * sv] != root) rc[r] = 2;
  }
#pragma omp parallel for schedule(static, 1 << 16) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t i = 0; i < m; ++i) {
    uint32_t a, b;
    get_pair(ps, i, &a, &b);
    if (a == b) continue;
    const int32_t u = (int32_t)a, v = (int32_t)b;
    if (has_nbr) {
      has_nbr[u] = 1;
      has_nbr[v] = 1;
    }
    for (int32_t r = 0; r < R; ++r) {
      if (rc[r] == 1 || rc[r] == 2) continue;
      const int64_t ou = r * sr + (int64_t)u * sv, ov = r * sr + (int64_t)v * sv;
      const int32_t lu = level[ou], lv = level[ov];
      if ((lu >= 0) != (lv >= 0)) {
        note_violation(&rc[r], &bad[r], 4, lu >= 0 ? u : v);
        continue;
      }
      if (lu < 0) continue;
      if (lu - lv > 1 || lv - lu > 1) {
        note_violation(&rc[r], &bad[r], 3, u);
        continue;
      }
      if (lu == lv - 1) __atomic_store_n(&up[ov], 1, __ATOMIC_RELAXED);
      if (lv == lu - 1) __atomic_store_n(&up[ou], 1, __ATOMIC_RELAXED);
      if (parent) {
        if (parent[ov] == u) __atomic_store_n(&confirmed[ov], 1, __ATOMIC_RELAXED);
        if (parent[ou] == v) __atomic_store_n(&confirmed[ou], 1, __ATOMIC_RELAXED);
      }
      if (canon) {
        if (lu == lv - 1) atomic_min_i32(&canon[ov], u);
        if (lv == lu - 1) atomic_min_i32(&canon[ou], v);
      }
    }
  }
  /* vertex rules, in increasing v for each root (the first failure is kept);
     the loop order follows the layout so that memory is read in order */
  if (vertex_major) {
    for (int64_t v = 0; v < n; ++v)
      for (int32_t r = 0; r < R; ++r)
        if (!rc[r] && (rc[r] = vertex_rule(r * sr + v * sv, v, roots[r], n, level, parent, up, confirmed,
                                           r * sr, sv)))
          bad[r] = v;
  } else {
    for (int32_t r = 0; r < R; ++r)
      for (int64_t v = 0; v < n && !rc[r]; ++v)
        if ((rc[r] = vertex_rule(r * sr + v * sv, v, roots[r], n, level, parent, up, confirmed, r * sr, sv)))
          bad[r] = v;
  }
  int32_t failed = 0;
  for (int32_t r = 0; r < R; ++r) {
    const int32_t root = roots[r];
    if (canon && !rc[r]) canon[r * sr + (int64_t)root * sv] = root;
    failed += rc[r] ? 1 : 0;
  }
  free(confirmed);
  free(up);
  return failed;
}

/* Streaming check of one BFS on the R-MAT graph of gen.h (see check_stream_core). */
int32_t oracle_check_bfs_rmat_stream(int scale, int64_t m, uint32_t t_a, uint32_t t_ab, uint32_t t_abc,
                                     uint64_t seed, int32_t root, const int32_t* level,
                                     const int32_t* parent, int32_t* canon, uint8_t* has_nbr,
                                     int32_t n_threads, int64_t* bad) {
  const pair_source ps = {0, scale, t_a, t_ab, t_abc, gen_key_pairs(seed), gen_key_perm(seed), NULL, NULL};
  int32_t rc = 0;
  check_stream_core(&ps, (int64_t)1 << scale, m, 1, &root, level, parent, canon, has_nbr, n_threads, &rc, bad, 0);
  return rc;
}

/* Streaming check of R BFS results on the R-MAT graph of gen.h (vertex_major: layout of the per-root arrays). */
int32_t oracle_check_bfs_rmat_stream_multi(int scale, int64_t m, uint32_t t_a, uint32_t t_ab, uint32_t t_abc,
                                           uint64_t seed, int32_t R, const int32_t* roots, const int32_t* level,
                                           const int32_t* parent, int32_t* canon, int32_t n_threads, int32_t* rc,
                                           int64_t* bad, int32_t vertex_major) {
  const pair_source ps = {0, scale, t_a, t_ab, t_abc, gen_key_pairs(seed), gen_key_perm(seed), NULL, NULL};
  return check_stream_core(&ps, (int64_t)1 << scale, m, R, roots, level, parent, canon, NULL, n_threads, rc, bad,
                           vertex_major);
}

/* Streaming check of R BFS results on the graph of m pairs held in src/dst. */
int32_t oracle_check_bfs_pairs_multi(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int32_t R,
                                     const int32_t* roots, const int32_t* level, const int32_t* parent,
                                     int32_t* canon, uint8_t* has_nbr, int32_t n_threads, int32_t* rc,
                                     int64_t* bad, int32_t vertex_major) {
  const pair_source ps = {1, 0, 0, 0, 0, 0, 0, src, dst};
  return check_stream_core(&ps, n, m, R, roots, level, parent, canon, has_nbr, n_threads, rc, bad, vertex_major);
}
