// Query server: continuous batching of single-root BFS queries over several
// resident graphs.
//
// Every added graph gets lane groups (64- or 128-lane bit-parallel
// traversals, see msbfs.cu), each on its own CUDA stream, so the work of different graphs
// and groups overlaps on the device. A scheduler thread runs the loop:
//   1. launch the direction switch of every group that holds or awaits
//      queries, with an asynchronous copy of its control block;
//   2. for each group, once its copy has landed: lanes whose frontier is
//      empty have finished; their levels are written into the queries'
//      outputs (flush with release, which frees the lanes), then waiting
//      queries of that graph are admitted into free lanes (seeded at the
//      current iteration, so lanes join a traversal already in flight), and
//      the kernels of the next level are launched;
//   3. queries whose output copies have completed (CUDA events) become
//      visible to dobfs_serve_poll.
// Admission takes a free lane and, for queries whose output is host memory,
// a device staging buffer of n int32 within the server's device-memory
// budget; new groups are created while queries wait and the budget allows.
// Every query's levels are those of a lone BFS from its root: lanes never
// interact, so a result is the same alone and in any mix.
#include <time.h>

#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "msbfs.cuh"

namespace dobfs {
namespace {

int64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

enum QState { kQueued = 0, kRunning = 1, kFlushing = 2, kDone = 3, kFailed = 4 };

struct Engine;

struct Query {
  uint64_t ticket = 0;
  int32_t gid = 0;
  int32_t root = 0;
  int32_t* out = nullptr;
  bool host_out = false;
  int64_t t_submit = 0, t_admit = 0, t_done = 0;
  int state = kQueued;
  int status = DOBFS_PENDING;
  int32_t start_iter = 0;
  int32_t levels = 0;
  DevBuf stage;  // device copy of the output when out is host memory
  cudaEvent_t ev = nullptr;
  int32_t* levels_h = nullptr;  // pinned slot the single-source path writes the level count to
  Engine* ss_engine = nullptr;  // set while the query runs on its engine's single-source path
};

struct Group {
  MsGroup* ms = nullptr;
  cudaStream_t stream = nullptr;
  MsCtl* hctl = nullptr;  // pinned
  Query* lane_q[kMsLanes] = {};
  LaneMask all = 0;   // the group's lanes (64 per mask word)
  LaneMask busy = 0;  // lanes holding a query
  bool in_flight = false;  // a switch and its control-block copy are queued
  cudaEvent_t ctl_ev = nullptr;
  int32_t cohort_iter = 0;  // iteration at which the group last went from idle to busy
  LaneMask finished = 0;    // lanes done but not yet flushed
  int32_t finish_iter[kMsLanes] = {};
  int64_t bytes = 0;
};

struct Engine {
  dobfs_graph* g = nullptr;
  std::vector<Group*> groups;
  std::deque<Query*> pending;
  // single-source path: lone queries run back to back as dobfs_run on this stream
  cudaStream_t ss_stream = nullptr;
  int32_t* ss_levels = nullptr;  // pinned ring of level counts
  int ss_next = 0;
  int ss_inflight = 0;
};
constexpr int kSsRing = 1024;

}  // namespace
}  // namespace dobfs

using namespace dobfs;

struct dobfs_server {
  dobfs_serve_opts opts;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::thread th;
  bool stop = false;
  std::vector<Engine*> engines;
  std::deque<Query*> inbox;
  std::unordered_map<uint64_t, Query*> queries;
  std::vector<Query*> flushing;
  std::list<Query*> done_list;  // finished and not yet polled or collected
  uint64_t next_ticket = 1;
  int64_t budget = 0;
  int64_t reserved = 0;
  int fatal = DOBFS_OK;
  std::string fatal_msg;
  int64_t iterations = 0, completed = 0, groups_created = 0;
  int64_t cohorts = 0, lanes_admitted = 0, group_steps = 0, single_source = 0;  // scheduler thread writes
  bool waiting_gpu = false;  // scheduler thread only: some group's switch is still running
};

namespace dobfs {
namespace {

int64_t group_bytes(const dobfs_server* S, const dobfs_graph* g) { return ms_group_bytes(g, S->opts.lane_words); }

// Creates a lane group on engine e (scheduler thread, or add_graph).
int add_group(dobfs_server* S, Engine* e) {
  Group* G = new (std::nothrow) Group();
  if (!G) return set_error(DOBFS_ERR_OOM, "host allocation failed");
  int rc = DOBFS_OK;
  if (cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void**)&G->hctl, sizeof(MsCtl)) != cudaSuccess ||
      cudaEventCreateWithFlags(&G->ctl_ev, cudaEventDisableTiming) != cudaSuccess) {
    rc = set_error(DOBFS_ERR_CUDA, "stream or pinned allocation failed");
  }
  if (rc == DOBFS_OK) rc = ms_group_create(e->g, G->stream, S->opts.lane_words, &G->ms);
  G->all = S->opts.lane_words == 2 ? ~(LaneMask)0 : (lane_bit(kMsWordLanes) - 1);
  if (rc == DOBFS_OK) {
    dobfs_run_opts o;
    dobfs_run_opts_init(&o);
    o.alpha = S->opts.alpha;
    o.beta = S->opts.beta;
    o.direction = S->opts.direction;
    rc = ms_group_reset(G->ms, o);
  }
  if (rc != DOBFS_OK) {
    if (G->ms) ms_group_destroy(G->ms);
    if (G->hctl) cudaFreeHost(G->hctl);
    if (G->ctl_ev) cudaEventDestroy(G->ctl_ev);
    if (G->stream) cudaStreamDestroy(G->stream);
    delete G;
    return rc;
  }
  G->bytes = group_bytes(S, e->g);
  e->groups.push_back(G);
  return DOBFS_OK;
}

void fail_all(dobfs_server* S, int rc, const char* msg) {
  std::lock_guard<std::mutex> lk(S->mu);
  S->fatal = rc;
  S->fatal_msg = msg;
  for (auto& kv : S->queries)
    if (kv.second->state != kDone) {
      kv.second->state = kFailed;
      kv.second->status = rc;
    }
}

// One pass of the scheduler over every group. Returns true if any group did work.
bool schedule_once(dobfs_server* S) {
  std::vector<Engine*> engines;  // add_graph may append concurrently: work on a copy
  {
    std::lock_guard<std::mutex> lk(S->mu);
    while (!S->inbox.empty()) {
      Query* q = S->inbox.front();
      S->inbox.pop_front();
      S->engines[q->gid]->pending.push_back(q);
    }
    engines = S->engines;
  }
  bool work = false;
  S->waiting_gpu = false;
  // Light load: a few waiting queries (device outputs) run as single-source
  // BFS on the engine's own stream, back to back with no host wait, as long
  // as that path's backlog is short; a longer queue is left to the lane
  // groups, whose cohorts amortise a traversal over many queries.
  for (Engine* e : engines) {
    while (!e->pending.empty() && (int)e->pending.size() <= S->opts.ss_max && e->ss_inflight < S->opts.ss_backlog &&
           !e->pending.front()->host_out) {
      Query* q = e->pending.front();
      e->pending.pop_front();
      dobfs_run_opts o;
      dobfs_run_opts_init(&o);  // single-source defaults (the lane groups' alpha suits many lanes)
      o.stream = (void*)e->ss_stream;
      int rc = dobfs_run(e->g, q->root, q->out, nullptr, &o, nullptr);
      q->levels_h = e->ss_levels + (e->ss_next++ % kSsRing);
      if (rc == DOBFS_OK) rc = graph_levels_async(e->g, q->levels_h, e->ss_stream);
      if (rc == DOBFS_OK && cudaEventRecord(q->ev, e->ss_stream) != cudaSuccess) rc = DOBFS_ERR_CUDA;
      if (rc != DOBFS_OK) {
        fail_all(S, rc, dobfs_last_error());
        return false;
      }
      q->t_admit = now_ns();
      q->state = kFlushing;
      q->ss_engine = e;
      e->ss_inflight += 1;
      S->single_source += 1;
      work = true;
      std::lock_guard<std::mutex> lk(S->mu);
      S->flushing.push_back(q);
    }
  }
  // Each group advances on its own: a group whose control block has landed
  // (its event has fired) is finished, admitted and relaunched; the others
  // are left running. A group's next switch is queued right behind its
  // level kernels, so its stream never waits for the host.
  for (Engine* e : engines) {
    dobfs_graph* g = e->g;
    for (Group* G : e->groups) {
      if (!G->in_flight) {
        if (!G->busy) {
          // an idle group starts a cohort once a full group of queries waits or
          // the oldest waiting query has waited gather_us
          if (e->pending.empty()) continue;
          const bool full = e->pending.size() >= (size_t)(kMsWordLanes * S->opts.lane_words);
          const bool old = now_ns() - e->pending.front()->t_submit >= (int64_t)S->opts.gather_us * 1000;
          if (!full && !old) {
            S->waiting_gpu = true;  // poll again shortly
            continue;
          }
        }
        if (ms_group_switch_async(G->ms, G->hctl) != DOBFS_OK ||
            cudaEventRecord(G->ctl_ev, G->stream) != cudaSuccess) {
          fail_all(S, DOBFS_ERR_CUDA, dobfs_last_error());
          return false;
        }
        G->in_flight = true;
        work = true;
        continue;
      }
      const cudaError_t evs = cudaEventQuery(G->ctl_ev);
      if (evs == cudaErrorNotReady) {
        S->waiting_gpu = true;
        continue;
      }
      if (evs != cudaSuccess) {
        fail_all(S, DOBFS_ERR_CUDA, "server stream failed");
        return false;
      }
      G->in_flight = false;
      work = true;
      MsCtl c = *G->hctl;
      if (c.bc_site) {
        fail_all(S, DOBFS_ERR_BOUNDS, bounds_site_name(c.bc_site));
        return false;
      }
      // lanes whose frontier emptied; each flush is a pass over the whole
      // graph, so finished lanes are flushed together: when the group has no
      // live lane left, or once the oldest has waited flush_delay levels
      const LaneMask live = lanes_of(c.live, G->ms->words);
      const LaneMask done_now = G->busy & ~live & ~G->finished;
      for (int i = 0; i < kMsLanes; ++i)
        if ((done_now >> i) & 1) G->finish_iter[i] = c.iter;
      G->finished |= done_now;
      bool flush_now = G->finished && (live == 0 || S->opts.flush_delay <= 0);
      for (int i = 0; i < kMsLanes && G->finished && !flush_now; ++i)
        if (((G->finished >> i) & 1) && c.iter - G->finish_iter[i] >= S->opts.flush_delay) flush_now = true;
      const LaneMask finished = flush_now ? G->finished : 0;
      if (finished) {
        int32_t* outs[kMsLanes] = {};
        int32_t starts[kMsLanes] = {};
        for (int i = 0; i < kMsLanes; ++i)
          if ((finished >> i) & 1) {
            Query* q = G->lane_q[i];
            outs[i] = q->host_out ? q->stage.as<int32_t>() : q->out;
            starts[i] = q->start_iter;
          }
        int rc = ms_group_flush(G->ms, finished, outs, starts, true);
        for (int i = 0; i < kMsLanes && rc == DOBFS_OK; ++i)
          if ((finished >> i) & 1) {
            Query* q = G->lane_q[i];
            if (q->host_out && cudaMemcpyAsync(q->out, q->stage.ptr, sizeof(int32_t) * (size_t)g->n,
                                               cudaMemcpyDeviceToHost, G->stream) != cudaSuccess)
              rc = DOBFS_ERR_CUDA;
            q->levels = G->finish_iter[i] - q->start_iter;
            if (rc == DOBFS_OK && cudaEventRecord(q->ev, G->stream) != cudaSuccess) rc = DOBFS_ERR_CUDA;
            q->state = kFlushing;
            G->lane_q[i] = nullptr;
            std::lock_guard<std::mutex> lk(S->mu);
            S->flushing.push_back(q);
          }
        if (rc != DOBFS_OK) {
          fail_all(S, rc, "flush failed");
          return false;
        }
        G->busy &= ~finished;
        G->finished = 0;
        if (G->busy == 0) {
          // every lane released: restart the iteration count (few discovery planes)
          if (ms_group_rebase(G->ms) != DOBFS_OK) {
            fail_all(S, DOBFS_ERR_CUDA, dobfs_last_error());
            return false;
          }
          c.iter = 0;
          if (c.n_planes > 4) c.n_planes = 4;
          G->hctl->iter = 0;
        }
      }
      // admission into free lanes: an idle group starts a new cohort; a busy
      // group takes more lanes only within join_window levels of its
      // cohort's start and at light levels (small union frontier). Lanes of
      // one cohort then reach their wide middle levels together, so one
      // bottom-up step serves all of them; queries arriving later go to
      // another group of the graph (created while the budget allows).
      int32_t lanes[kMsLanes], roots[kMsLanes];
      int k = 0;
      const bool idle = (G->busy == 0);
      if (idle) G->cohort_iter = c.iter;
      const bool light = S->opts.admit_div <= 0 || c.n_f * (int64_t)S->opts.admit_div < g->n;
      const bool can_join = (G->busy == 0) || (light && c.iter - G->cohort_iter <= S->opts.join_window);
      LaneMask freel = can_join ? (G->all & ~G->busy) : 0;
      while (freel && !e->pending.empty()) {
        Query* q = e->pending.front();
        const int64_t need = q->host_out ? (int64_t)sizeof(int32_t) * g->n : 0;
        {
          std::lock_guard<std::mutex> lk(S->mu);
          if (S->reserved + need > S->budget) break;  // waits for memory to free up
          S->reserved += need;
        }
        if (need && q->stage.alloc((size_t)need, G->stream) != DOBFS_OK) {
          std::lock_guard<std::mutex> lk(S->mu);
          S->reserved -= need;
          break;
        }
        e->pending.pop_front();
        const int lane = first_lane(freel);
        freel &= freel - 1;
        q->start_iter = c.iter;
        q->t_admit = now_ns();
        q->state = kRunning;
        G->lane_q[lane] = q;
        G->busy |= lane_bit(lane);
        lanes[k] = lane;
        roots[k] = q->root;
        ++k;
      }
      if (k) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->lanes_admitted += k;
        S->cohorts += idle ? 1 : 0;
      }
      if (k && ms_group_seed(G->ms, k, lanes, roots) != DOBFS_OK) {
        fail_all(S, DOBFS_ERR_CUDA, dobfs_last_error());
        return false;
      }
      if (live || k) {
        S->group_steps += 1;
        // lanes seeded after the switch start top-down: a bottom-up step they
        // join runs as a step of both kinds
        if (ms_group_case_async(G->ms, (k && c.step_case == 1) ? 2 : c.step_case) != DOBFS_OK) {
          fail_all(S, DOBFS_ERR_CUDA, dobfs_last_error());
          return false;
        }
      }
      if (G->busy || !e->pending.empty()) {  // next level's switch, queued behind the kernels
        if (ms_group_switch_async(G->ms, G->hctl) != DOBFS_OK ||
            cudaEventRecord(G->ctl_ev, G->stream) != cudaSuccess) {
          fail_all(S, DOBFS_ERR_CUDA, dobfs_last_error());
          return false;
        }
        G->in_flight = true;
      }
    }
    // another group while queries wait, lanes are full and memory allows
    bool all_full = true;  // no group can take a waiting query now
    for (Group* G : e->groups) {
      const bool light = S->opts.admit_div <= 0 || G->hctl->n_f * (int64_t)S->opts.admit_div < g->n;
      const bool can_join =
          (G->busy == 0) || (light && G->hctl->iter - G->cohort_iter <= S->opts.join_window && (G->all & ~G->busy) != 0);
      all_full = all_full && !can_join;
    }
    if (!e->pending.empty() && all_full && (int)e->groups.size() < S->opts.max_groups_per_graph) {
      const int64_t gb = group_bytes(S, g);
      bool ok;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        ok = S->reserved + gb <= S->budget;
        if (ok) S->reserved += gb;
      }
      if (ok) {
        if (add_group(S, e) == DOBFS_OK) {
          S->groups_created += 1;
        } else {
          std::lock_guard<std::mutex> lk(S->mu);
          S->reserved -= gb;
        }
      }
    }
  }
  // 3. completions (staging buffers are released after the lock is dropped)
  std::vector<DevBuf> to_free;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t i = 0; i < S->flushing.size();) {
      Query* q = S->flushing[i];
      const cudaError_t st = cudaEventQuery(q->ev);
      if (st == cudaErrorNotReady) {
        ++i;
        continue;
      }
      q->t_done = now_ns();
      q->state = (st == cudaSuccess) ? kDone : kFailed;
      if (q->ss_engine) {
        q->levels = *q->levels_h;
        q->ss_engine->ss_inflight -= 1;
        q->ss_engine = nullptr;
      }
      q->status = (st == cudaSuccess) ? DOBFS_OK : DOBFS_ERR_CUDA;
      if (q->stage.ptr) {
        S->reserved -= (int64_t)q->stage.bytes;
        to_free.push_back(std::move(q->stage));
      }
      S->completed += 1;
      S->done_list.push_back(q);
      S->flushing[i] = S->flushing.back();
      S->flushing.pop_back();
      work = true;
    }
  }
  S->iterations += work ? 1 : 0;
  return work;
}

void scheduler(dobfs_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop) break;
      if (S->fatal != DOBFS_OK) {
        S->cv.wait_for(lk, std::chrono::milliseconds(10));
        continue;
      }
    }
    const bool work = schedule_once(S);
    if (!work) {
      if (S->waiting_gpu) {  // some group's level is running: poll again shortly
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        continue;
      }
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop) break;
      if (S->inbox.empty() && S->flushing.empty()) S->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
}

}  // namespace
}  // namespace dobfs

extern "C" {

int dobfs_serve_opts_init(dobfs_serve_opts* o) {
  if (!o) return set_error(DOBFS_ERR_INVALID, "opts is NULL");
  memset(o, 0, sizeof(*o));
  o->max_device_bytes = 0;
  o->groups_per_graph = 1;
  o->max_groups_per_graph = 1;
  o->alpha = DOBFS_BATCH_ALPHA;
  o->beta = 24;
  o->direction = DOBFS_DIR_AUTO;
  o->admit_div = 64;
  o->join_window = 1;
  o->flush_delay = 3;
  o->gather_us = 2000;
  o->ss_max = 2;
  o->ss_backlog = 4;
  o->lane_words = 2;
  return DOBFS_OK;
}

int dobfs_serve_create(const dobfs_serve_opts* opts, dobfs_server** out) {
  clear_error();
  if (!out) return set_error(DOBFS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  dobfs_serve_opts o;
  dobfs_serve_opts_init(&o);
  if (opts) o = *opts;
  if (o.groups_per_graph < 1 || o.max_groups_per_graph < o.groups_per_graph || o.alpha < 1 || o.beta < 1 ||
      o.direction < 0 || o.direction > DOBFS_DIR_RANDOM || o.max_device_bytes < 0 || o.admit_div < 0 ||
      o.join_window < 0 || o.flush_delay < 0 || o.gather_us < 0 || o.ss_max < 0 || o.ss_backlog < 0 ||
      o.lane_words < 1 || o.lane_words > kMsMaxWords)
    return set_error(DOBFS_ERR_INVALID, "bad server options");
  dobfs_server* S = new (std::nothrow) dobfs_server();
  if (!S) return set_error(DOBFS_ERR_OOM, "host allocation failed");
  S->opts = o;
  cudaGetDevice(&S->device);
  if (o.max_device_bytes > 0) {
    S->budget = o.max_device_bytes;
  } else {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete S;
      return set_error(DOBFS_ERR_CUDA, "cudaMemGetInfo failed");
    }
    S->budget = (int64_t)(0.9 * (double)fr);
  }
  S->th = std::thread(scheduler, S);
  *out = S;
  return DOBFS_OK;
}

int dobfs_serve_add_graph(dobfs_server* S, dobfs_graph* g, int32_t* gid) {
  clear_error();
  if (!S || !g || !gid) return set_error(DOBFS_ERR_INVALID, "NULL argument");
  Engine* e = new (std::nothrow) Engine();
  if (!e) return set_error(DOBFS_ERR_OOM, "host allocation failed");
  e->g = g;
  if (cudaStreamCreateWithFlags(&e->ss_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void**)&e->ss_levels, sizeof(int32_t) * kSsRing) != cudaSuccess) {
    if (e->ss_stream) cudaStreamDestroy(e->ss_stream);
    delete e;
    return set_error(DOBFS_ERR_CUDA, "stream or pinned allocation failed");
  }
  const int64_t gb = group_bytes(S, g) * S->opts.groups_per_graph;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->reserved + gb > S->budget) {
      cudaStreamDestroy(e->ss_stream);
      cudaFreeHost(e->ss_levels);
      delete e;
      return set_error(DOBFS_ERR_BUSY, "device-memory budget too small for the graph's lane groups");
    }
    S->reserved += gb;
  }
  for (int i = 0; i < S->opts.groups_per_graph; ++i) {
    const int rc = add_group(S, e);
    if (rc != DOBFS_OK) {
      for (Group* G : e->groups) {
        ms_group_destroy(G->ms);
        cudaFreeHost(G->hctl);
        cudaEventDestroy(G->ctl_ev);
        cudaStreamDestroy(G->stream);
        delete G;
      }
      cudaStreamDestroy(e->ss_stream);
      cudaFreeHost(e->ss_levels);
      delete e;
      std::lock_guard<std::mutex> lk(S->mu);
      S->reserved -= gb;
      return rc;
    }
  }
  std::lock_guard<std::mutex> lk(S->mu);
  *gid = (int32_t)S->engines.size();
  S->engines.push_back(e);
  return DOBFS_OK;
}

int dobfs_serve_submit(dobfs_server* S, int32_t gid, int32_t root, int32_t* level_out, int32_t* parent_out,
                       uint64_t* ticket) {
  clear_error();
  if (!S || !level_out || !ticket) return set_error(DOBFS_ERR_INVALID, "server, level_out and ticket are required");
  if (parent_out) return set_error(DOBFS_ERR_INVALID, "served queries return levels only (parent_out must be NULL)");
  Query* q = new (std::nothrow) Query();
  if (!q) return set_error(DOBFS_ERR_OOM, "host allocation failed");
  q->host_out = !is_device_ptr(level_out);
  if (cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming) != cudaSuccess) {
    delete q;
    return set_error(DOBFS_ERR_CUDA, "event creation failed");
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->fatal != DOBFS_OK) {
    cudaEventDestroy(q->ev);
    delete q;
    return set_error(S->fatal, "server failed: %s", S->fatal_msg.c_str());
  }
  if (gid < 0 || gid >= (int32_t)S->engines.size()) {
    cudaEventDestroy(q->ev);
    delete q;
    return set_error(DOBFS_ERR_INVALID, "unknown graph id %d", gid);
  }
  if (root < 0 || root >= S->engines[gid]->g->n) {
    cudaEventDestroy(q->ev);
    delete q;
    return set_error(DOBFS_ERR_INVALID, "root %d out of range", root);
  }
  q->gid = gid;
  q->root = root;
  q->out = level_out;
  q->t_submit = now_ns();
  q->ticket = S->next_ticket++;
  S->queries[q->ticket] = q;
  S->inbox.push_back(q);
  *ticket = q->ticket;
  S->cv.notify_one();
  return DOBFS_OK;
}

int dobfs_serve_poll(dobfs_server* S, uint64_t ticket, dobfs_query_result* res) {
  if (!S) return set_error(DOBFS_ERR_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->queries.find(ticket);
  if (it == S->queries.end()) return set_error(DOBFS_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
  Query* q = it->second;
  if (q->state != kDone && q->state != kFailed) return DOBFS_PENDING;
  if (res) {
    res->status = q->status;
    res->levels = q->levels;
    res->submit_ns = q->t_submit;
    res->admit_ns = q->t_admit;
    res->done_ns = q->t_done;
    res->latency_ns = q->t_done - q->t_submit;
  }
  const int st = q->status;
  S->done_list.remove(q);
  cudaEventDestroy(q->ev);
  delete q;
  S->queries.erase(it);
  return st == DOBFS_OK ? DOBFS_OK : set_error(st, "query failed");
}

int dobfs_serve_collect(dobfs_server* S, uint64_t* tickets, dobfs_query_result* results, int32_t max_results,
                        int32_t* n_out) {
  if (!S || !tickets || !results || !n_out || max_results < 0) return set_error(DOBFS_ERR_INVALID, "bad arguments");
  std::lock_guard<std::mutex> lk(S->mu);
  int32_t n = 0;
  for (auto it = S->done_list.begin(); it != S->done_list.end() && n < max_results;) {
    Query* q = *it;
    tickets[n] = q->ticket;
    results[n].status = q->status;
    results[n].levels = q->levels;
    results[n].submit_ns = q->t_submit;
    results[n].admit_ns = q->t_admit;
    results[n].done_ns = q->t_done;
    results[n].latency_ns = q->t_done - q->t_submit;
    ++n;
    S->queries.erase(q->ticket);
    cudaEventDestroy(q->ev);
    delete q;
    it = S->done_list.erase(it);
  }
  *n_out = n;
  return DOBFS_OK;
}

int dobfs_serve_get_stats(dobfs_server* S, dobfs_serve_stats* st) {
  if (!S || !st) return set_error(DOBFS_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  st->iterations = S->iterations;
  st->completed = S->completed;
  st->in_flight = (int64_t)S->queries.size();
  st->groups_created = S->groups_created;
  st->reserved_bytes = S->reserved;
  st->budget_bytes = S->budget;
  st->cohorts = S->cohorts;
  st->lanes_admitted = S->lanes_admitted;
  st->group_steps = S->group_steps;
  st->single_source = S->single_source;
  return S->fatal;
}

int dobfs_serve_destroy(dobfs_server* S) {
  if (!S) return DOBFS_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->th.joinable()) S->th.join();
  for (Engine* e : S->engines) {
    for (Group* G : e->groups) {
      cudaStreamSynchronize(G->stream);
      ms_group_destroy(G->ms);
      cudaFreeHost(G->hctl);
      cudaEventDestroy(G->ctl_ev);
      cudaStreamDestroy(G->stream);
      delete G;
    }
    cudaStreamSynchronize(e->ss_stream);
    {
      // the graph's next run must not wait on a stream that is about to go away
      std::lock_guard<std::mutex> lk(e->g->mu);
      if (e->g->last_stream == e->ss_stream) e->g->last_stream = nullptr;
    }
    cudaStreamDestroy(e->ss_stream);
    cudaFreeHost(e->ss_levels);
    delete e;
  }
  for (auto& kv : S->queries) {
    cudaEventDestroy(kv.second->ev);
    delete kv.second;
  }
  delete S;
  return DOBFS_OK;
}

}  // extern "C"
