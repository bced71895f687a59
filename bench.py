"""Benchmark: single-source direction-optimized BFS, GTEPS on R-MAT scale 28.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat28|rmat22|rmat16|chunglu26]
                    [--impl ours|reference]

One step = one BFS from one seeded root on the resident graph: status init,
the device-driven level loop (top-down / bottom-up steps and the switch),
and the outputs (level and parent per vertex, original IDs) written to device
buffers. GTEPS per root = undirected edges in the root's component / device
time (CUDA events on the launching stream); the reported value is the
harmonic mean over the K timed roots (Graph500 convention). The scale-28
graph (~48 GB resident) is far larger than L2, so no flush is needed between
steps. With N > 1 (torchrun) every rank runs independent replicas on its own
GPU: BFS from a single root does not shard without a per-level exchange, so
the job's value is the sum of the ranks' rates measured over the max time.

Workloads: rmat28 (default, the headline), rmat22 (int64 offsets), rmat16
(no renumbering, int32 offsets) and chunglu26 (Chung-Lu power-law graph,
2^26 vertices, exponent 2.1, mean degree 35); batched and served BFS are
measured with the default workload only.

Also reported: the roofline of each step kind (top-down, bottom-up, mixed;
the dominant one in `roofline` itself), measured per level with CUDA events
in host-driven mode on a fixed sample of 16 roots, the same whatever
--steps and --warmup are, so that an ncu capture of this command measures
the same launches; the DRAM traffic per bottom-up level, scaled from the
committed ncu capture of a smaller graph when the kernel sources still
match it; an end-to-end number through the C ABI with host (pinned) output
buffers; the batched BFS against its algorithmic bytes; the CPU oracle on a
bounded sample of the same workload; SM clocks sampled during the timed
region; and the number of kernels launched. With --tune the direction
policy and degree-bin cutoffs are first tuned on 8 other roots
(autotune.py) and the timed pass uses the tuned options.
"""
from __future__ import annotations

import argparse
import collections
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GTEPS at R-MAT scale 28; batched BFS/s and p50/p99 latency vs serial BFS"

# name -> (generator, size, build flags by name, timed roots by default)
WORKLOADS = {
    "rmat16": ("rmat", 16, ("",), 16),
    "rmat22": ("rmat", 22, ("REINDEX", "OFFSETS64"), 64),
    "rmat28": ("rmat", 28, ("REINDEX",), 64),
    "chunglu26": ("chunglu", 26, ("REINDEX",), 64),
}
DEFAULT_WORKLOAD = "rmat28"

# the oracle's sample on graphs it cannot traverse in full on one core in the
# time allowed: the FIFO BFS stopped after this many adjacency entries per root
CPU_SAMPLE_ENTRIES = 1 << 29
REF_STEP_ENTRIES = 1 << 28


def workload_name(kind: str, size: int) -> str:
    """The graph's identity (the same for the oracle and the library, whatever
    the library's internal layout)."""
    return "rmat-s%d-ef16" % size if kind == "rmat" else "chunglu-2^%d-g2.1-mean35-max2^20" % size


def make_spec(inputs, kind: str, size: int):
    return inputs.rmat(size) if kind == "rmat" else inputs.chunglu(size)


def host_info() -> dict:
    """CPU model, logical cores and memory of this host (for the CPU baseline)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    mem_gb = avail_gb = None
    try:
        with open("/proc/meminfo") as f:
            kv = {l.split(":")[0]: l.split(":")[1].strip() for l in f}
        mem_gb = int(kv["MemTotal"].split()[0]) / 1e6
        avail_gb = int(kv["MemAvailable"].split()[0]) / 1e6
    except (OSError, KeyError, ValueError):
        pass
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"cpu": model, "cores": cores, "mem_gb": mem_gb, "mem_available_gb": avail_gb}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


KERNEL_SOURCES = ("paper_1503_04359_b300/csrc/bfs.cu", "paper_1503_04359_b300/csrc/graph.cuh",
                  "paper_1503_04359_b300/csrc/common.cuh")
TRAFFIC_PROFILE = "profiles/bu_step_rmat_s24.md"
STEP_NAMES = {0: "top-down", 1: "bottom-up", 2: "mixed"}
STEP_KERNELS = {0: "top-down step (k_td_bin + k_td_chunks [+ k_bu parent search])",
                1: "bottom-up step (k_bu + k_bu_long)",
                2: "mixed step (k_td_bin + k_td_chunks + k_bu + k_bu_long)"}


def kernel_sha256() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic():
    """The traffic record of the committed ncu summary (DRAM bytes and
    algorithmic bytes of the bottom-up levels of a capture on a graph small
    enough to capture with several metrics), if it was taken with the current
    kernel sources; else None."""
    try:
        with open(os.path.join(ROOT, TRAFFIC_PROFILE)) as f:
            m = re.search(r"<!-- traffic (\{.*?\}) -->", f.read(), re.S)
        rec = json.loads(m.group(1))
    except Exception:
        return None
    if rec.get("kernel_sha256") != kernel_sha256():
        return None
    return rec


def aggregate_ranks(dist, device, total_ms: float, total_edges: float) -> tuple[float, float]:
    """Whole-job GTEPS of independent replicas: the edges every rank traversed
    over the slowest rank's timed region (max over ranks). Returns (GTEPS, max ms)."""
    import torch
    t = torch.tensor([total_ms, total_edges], dtype=torch.float64, device=device)
    allt = [torch.zeros_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(allt, t)
    mx = max(float(x[0]) for x in allt)
    return sum(float(x[1]) for x in allt) / (mx * 1e-3) / 1e9, mx


def combine_batch(per_rank: list) -> dict:
    """Batched-BFS results of independent replicas (one per rank, each on its
    own GPU and graph copy): every batch size's roots over all ranks divided
    by the slowest rank's time; the rest from rank 0."""
    out = json.loads(json.dumps(per_rank[0]))
    ws = len(per_rank)
    seq_ms = max(r["sequential"]["ms"] for r in per_rank)
    out["sequential"]["ms"] = seq_ms
    out["sequential"]["roots"] = sum(r["sequential"]["roots"] for r in per_rank)
    out["sequential"]["roots_per_s"] = out["sequential"]["roots"] / (seq_ms * 1e-3)
    for b, x in out["batches"].items():
        ms = max(r["batches"][b]["ms"] for r in per_rank)
        x["ms"] = ms
        x["roots_per_s"] = ws * int(b) / (ms * 1e-3)
        x["speedup_vs_sequential"] = x["roots_per_s"] / out["sequential"]["roots_per_s"]
        x["gteps_est"] = sum(r["batches"][b]["gteps_est"] * r["batches"][b]["ms"] for r in per_rank) / ms
        rf = x.get("roofline")
        if rf:
            rf["alg_bytes"] = sum(r["batches"][b]["roofline"]["alg_bytes"] for r in per_rank)
            rf["achieved"] = rf["alg_bytes"] / (ms * 1e-3) / 1e9
            rf["peak"] = rf["peak"] * ws
            rf["frac"] = rf["achieved"] / rf["peak"]
    out["replicas"] = ws
    return out


def combine_serve(per_rank: list) -> dict:
    """Serving results of independent replicas (each rank serves its own
    Poisson stream on its own GPU): queries over all ranks divided by the
    longest span, latency percentiles over every rank's queries."""
    out = json.loads(json.dumps({k: v for k, v in per_rank[0].items() if k != "rates"}))
    out["rates"] = {}
    ws = len(per_rank)
    base_qps = sum(r["one_at_a_time"]["qps"] for r in per_rank)
    out["one_at_a_time"]["qps"] = base_qps
    for rate in per_rank[0]["rates"]:
        rs = [r["rates"][rate] for r in per_rank]
        lat = np.concatenate([np.asarray(x["_latencies_ms"]) for x in rs])
        q = sum(x["queries"] for x in rs)
        span = max(x["span_s"] for x in rs)
        out["rates"][rate] = {"queries": q, "offered_qps_per_replica": int(rate),
                              "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                              "mean_ms": float(lat.mean()), "achieved_qps": q / span, "span_s": span,
                              "vs_one_at_a_time": (q / span) / base_qps, "server": rs[0]["server"]}
    out["replicas"] = ws
    return out


def strip_private(res):
    """Drops the per-query latency lists (kept only for combining ranks)."""
    if isinstance(res, dict):
        return {k: strip_private(v) for k, v in res.items() if not k.startswith("_")}
    return res


def gpu_bus_id(torch, dev: int) -> str:
    """PCI bus id of CUDA device `dev` (as nvidia-smi and NVML name it), so the
    samplers read the GPU this process runs on whatever the visible-device mapping."""
    p = torch.cuda.get_device_properties(dev)
    return "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: str):
        self.gpu = gpu  # nvidia-smi -i accepts an index or a PCI bus id
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def nvml_energy_reader(bus_id: str):
    """A function returning the GPU's cumulative energy in mJ
    (nvmlDeviceGetTotalEnergyConsumption through the driver's NVML library,
    read only), or None where NVML or the counter is unavailable."""
    import ctypes
    try:
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByPciBusId_v2(bus_id.encode(), ctypes.byref(h)) != 0:
            return None
        mj = ctypes.c_ulonglong()

        def read():
            if lib.nvmlDeviceGetTotalEnergyConsumption(h, ctypes.byref(mj)) != 0:
                raise RuntimeError("NVML energy counter read failed")
            return int(mj.value)

        read()
        return read
    except (OSError, AttributeError, RuntimeError):
        return None


def energy_pass(torch, g, roots, level, parent, opts, teps, bus_id: str, seconds: float = 2.0):
    """Energy per BFS from the GPU's cumulative energy counter (NVML, read only),
    over repeated passes of the timed roots lasting about `seconds`; None if
    NVML is unavailable. MTEPS/W = traversed edges / joules / 1e6 (the
    paper's energy metric, Sec. 4)."""
    energy_mj = nvml_energy_reader(bus_id)
    if energy_mj is None:
        return None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for r in roots:
        g.run(int(r), level, parent, opts)
    e1.record()
    torch.cuda.synchronize()
    reps = max(1, int(seconds / max(1e-3, e0.elapsed_time(e1) * 1e-3)))
    torch.cuda.synchronize()
    mj0 = energy_mj()
    t0 = time.perf_counter()
    for _ in range(reps):
        for r in roots:
            g.run(int(r), level, parent, opts)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    mj1 = energy_mj()
    joules = (mj1 - mj0) * 1e-3
    edges = float(sum(teps)) * reps
    n = reps * len(roots)
    return {"bfs": n, "seconds": round(dt, 3), "joules_per_bfs": joules / n, "mean_power_w": joules / dt,
            "mteps_per_w": edges / joules / 1e6 if joules > 0 else None,
            "source": "NVML total energy counter (read only), graph-driven runs of the timed roots"}


def oracle_graph(inputs, oracle, kind: str, size: int, threads: int):
    """The workload's spec and the oracle's host CSR of it (threaded build)."""
    spec = make_spec(inputs, kind, size)
    if kind == "rmat":
        return spec, oracle.csr_from_rmat_par(spec, n_threads=threads)
    cdf = inputs.chunglu_cdf(spec)
    src, dst = inputs.chunglu_pairs(spec, cdf)
    g = oracle.csr_from_pairs_par(spec.n_vertices, src, dst, n_threads=threads)
    del src, dst
    return spec, g


def oracle_host_gb(kind: str, size: int) -> float:
    """Host memory the oracle's graph build and BFS need at peak (GB)."""
    n = 1 << size
    m = 16 * n if kind == "rmat" else int(n * 35 / 2)
    pairs = 0 if kind == "rmat" else 8 * m
    return (8 * m + 16 * n + 8 * n + pairs) / 1e9  # columns, offsets + cursors, level and parent


def oracle_timing(oracle, g, roots, limit):
    """Times the oracle's serial BFS (levels) from each root on one core:
    the full BFS (limit None) or the FIFO BFS stopped after `limit`
    adjacency entries. Returns (harmonic-mean GTEPS, seconds): TEPS =
    undirected edges traversed = entries read / 2 (for a full BFS, the edges
    of the root's component)."""
    rates, t_sum = [], 0.0
    for r in roots:
        t0 = time.perf_counter()
        if limit is None:
            lv, _, _ = oracle.bfs(g, int(r), want_parent=False)
            dt = time.perf_counter() - t0
            e = oracle.teps_edges(g, lv)
        else:
            _, read = oracle.bfs_partial(g, int(r), limit)
            dt = time.perf_counter() - t0
            e = read / 2.0
        t_sum += dt
        rates.append(e / dt / 1e9)
    return len(rates) / sum(1.0 / x for x in rates), t_sum, rates


def pick_oracle_size(kind: str, size: int, avail_gb) -> int:
    """The workload's size, or the largest smaller one of the same family whose
    oracle graph fits in the available host memory (with 15 % to spare)."""
    s = size
    while avail_gb is not None and s > 10 and oracle_host_gb(kind, s) * 1.15 > avail_gb:
        s -= 1
    return s


def cpu_baseline(workload: str, n_roots: int = 4, full: bool = False, all_cores: bool = False) -> dict:
    """The CPU oracle (serial FIFO BFS, levels, 1 thread) on the bench's own
    workload: full BFS from n_roots seeded roots where the graph is small
    enough, else (or unless `full`) the BFS of each root stopped after
    CPU_SAMPLE_ENTRIES adjacency entries. The oracle's graph is built by its
    threaded builder first (not timed). With all_cores, also roots/s of full
    BFS, one root per core on every core."""
    import dobfs_inputs as inputs
    import oracle

    kind, size, _, _ = WORKLOADS[workload]
    info = host_info()
    osize = pick_oracle_size(kind, size, info["mem_available_gb"])
    t0 = time.perf_counter()
    spec, g = oracle_graph(inputs, oracle, kind, osize, info["cores"] or 1)
    build_s = time.perf_counter() - t0
    deg = g.degrees()
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), g.n, n_roots, deg > 0)
    limit = None if (full or g.nnz <= 2 * CPU_SAMPLE_ENTRIES) else CPU_SAMPLE_ENTRIES
    hm, t_sum, rates = oracle_timing(oracle, g, roots, limit)
    what = ("full BFS" if limit is None else
            "BFS stopped after %d adjacency entries (of %d stored)" % (limit, g.nnz))
    sample = ("oracle serial FIFO BFS (levels), %d seeded roots on %s (%s; graph built by the oracle's threaded "
              "builder in %.0f s, not timed), %s, harmonic mean" %
              (n_roots, workload_name(kind, osize), "the bench's own graph" if osize == size else
               "the largest of its family that fits in host memory", build_s, what))
    out = {"value": hm, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample, "seconds": t_sum,
           "per_root_gteps": rates, "oracle_build_s": build_s, "host": info,
           "same_workload": osize == size}
    if all_cores:
        k = min(64, info["cores"] or 1)
        mroots = inputs.sample_roots(inputs.root_seed(spec.seed) ^ 0xA11C, g.n, k, deg > 0)
        t0 = time.perf_counter()
        oracle.bfs_many(g, mroots, want_parent=False, n_threads=info["cores"])
        dt = time.perf_counter() - t0
        out["all_cores"] = {"roots": k, "threads": info["cores"], "seconds": dt, "roots_per_s": k / dt,
                            "sample": "%d full serial BFS (levels), one per core, on %s" %
                                      (k, workload_name(kind, osize))}
    return out


def measure_batch(torch, inputs, dobfs, scale: int, peak: float, sizes=(64, 256, 1024), reps: int = 3,
                  rank: int = 0) -> dict:
    """Batched BFS (bit-parallel lane groups of 64 or 128 roots) against one-at-a-time runs on
    the same R-MAT graph: roots/s for batches of 64/256/1024 seeded roots and
    for 64 sequential single-source runs (levels only in both), with device
    time from CUDA events. Outputs stay on the device (1024 x n int32). Each
    batch's algorithmic bytes come from an untimed run with statistics (per
    step of a W-word lane group: 16 W per active vertex, 8 W + 4 per examined
    entry; plus 4 per level written), its roofline from the timed runs."""
    spec = inputs.rmat(scale)
    g = dobfs.rmat_graph(spec, flags=dobfs.DOBFS_GRAPH_REINDEX)
    n = g.n
    deg = g.degrees()
    roots = inputs.sample_roots((inputs.root_seed(spec.seed) ^ 0xBA7C) + rank * 0x1000, n, max(sizes), deg > 0)
    stream = torch.cuda.current_stream()
    opts = dobfs.make_opts(stream=stream)  # single-source defaults
    bopts = dobfs.make_opts(stream=stream, alpha=dobfs.DOBFS_BATCH_ALPHA)  # the batch default
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    teps = []
    for r in roots[:64]:
        teps.append(g.run(int(r), lv, None, opts, want_stats=True).teps_edges)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for r in roots[:64]:
        g.run(int(r), lv, None, opts)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    seq_rps = 64 / (seq_ms * 1e-3)
    out = torch.empty((max(sizes), n), dtype=torch.int32, device="cuda")
    res = {"workload": "rmat-s%d-ef16-reindex" % scale, "n_vertices": n, "n_entries": int(g.info.n_entries),
           "sequential": {"roots": 64, "ms": seq_ms, "roots_per_s": seq_rps,
                          "gteps": float(np.sum(teps)) / (seq_ms * 1e-3) / 1e9},
           "batches": {}}
    mean_teps = float(np.mean(teps))
    for b in sizes:
        rt = torch.from_numpy(np.ascontiguousarray(roots[:b])).cuda()
        bst = dobfs.dobfs_run_batch(g.handle, rt, out[:b], opts=bopts, want_stats=True)
        times = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0.record(stream)
            dobfs.dobfs_run_batch(g.handle, rt, out[:b], opts=bopts)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = float(np.median(times))
        rps = b / (ms * 1e-3)
        gbs = bst.alg_bytes / (ms * 1e-3) / 1e9
        res["batches"][str(b)] = {"ms": ms, "roots_per_s": rps, "speedup_vs_sequential": rps / seq_rps,
                                  "gteps_est": b * mean_teps / (ms * 1e-3) / 1e9,
                                  "levels": int(bst.levels), "edges_examined": int(bst.edges_examined),
                                  "roofline": {"bound": "hbm", "alg_bytes": int(bst.alg_bytes), "achieved": gbs,
                                               "peak": peak, "unit": "GB/s", "frac": gbs / peak}}
    del out
    g.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def measure_serve(torch, inputs, dobfs, scales=(18, 20, 22, 24, 26), rates=(2000, 5000, 10000, 20000, 50000),
                  seconds: float = 2.0, max_queries: int = 20000, out_gb: float = 120.0, min_slots: int = 256,
                  serve_opts=None, rank: int = 0) -> dict:
    """Open-loop serving: R-MAT graphs of the given scales resident, Poisson
    arrivals (seeded exponential gaps) at each rate, graph ids uniform, roots
    uniform over degree >= 1 vertices. Latency runs from the scheduled arrival
    to the completion the server reports (CLOCK_MONOTONIC), so a harness that
    falls behind its schedule is charged for it. Output buffers come from a
    per-graph pool of device slots: an even share of out_gb, at least
    min_slots (two full 128-lane cohorts: one running while the next gathers)
    and at most 1024 per graph; a query whose graph has no free slot waits in
    its graph's FIFO without holding up other graphs. The
    one-at-a-time baseline is the device time of single-source runs (levels
    only) averaged over the same mix."""
    graphs, pools, slots = [], [], []
    per_graph_bytes = out_gb * 1e9 / len(scales)
    base_ms = []
    for sc in scales:
        spec = inputs.rmat(sc)
        g = dobfs.rmat_graph(spec, flags=dobfs.DOBFS_GRAPH_REINDEX)
        deg = g.degrees()
        pool = inputs.sample_roots(inputs.root_seed(spec.seed) ^ 0x5E7E, g.n, 1024, deg > 0)
        k = int(min(1024, max(min_slots, per_graph_bytes // (4 * g.n))))
        slots.append(torch.empty((k, g.n), dtype=torch.int32, device="cuda"))
        lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
        ms = [g.run(int(r), lv, None, want_stats=True).device_ms for r in pool[:8]]
        base_ms.append(float(np.mean(ms[2:])))
        graphs.append(g)
        pools.append(pool)
    one_at_a_time_qps = 1000.0 / float(np.mean(base_ms))
    srv = dobfs.dobfs_serve_create(serve_opts if serve_opts is not None else dobfs.make_serve_opts())
    col = dobfs.Collector()
    res = {"workload": "rmat-s%s-ef16-reindex resident, gid uniform, Poisson arrivals" % "/".join(map(str, scales)),
           "one_at_a_time": {"mean_device_ms_per_graph": base_ms, "qps": one_at_a_time_qps}, "rates": {}}
    try:
        gids = [dobfs.dobfs_serve_add_graph(srv, g.handle) for g in graphs]
        for rate in rates:
            st0 = dobfs.dobfs_serve_get_stats(srv)
            n_q = int(max(200, min(max_queries, rate * seconds)))
            rng = np.random.default_rng(0xA11CE + rate + 7919 * rank)
            gaps = rng.exponential(1.0 / rate, n_q)
            which = rng.integers(0, len(graphs), n_q)
            ridx = rng.integers(0, 1024, n_q)
            free = [list(range(s.shape[0])) for s in slots]
            waiting = [collections.deque() for _ in graphs]  # arrived, no output slot yet (per graph)
            inflight = {}
            lat = []
            t0 = time.monotonic_ns() + 2_000_000
            sched = t0 + (np.cumsum(gaps) * 1e9).astype(np.int64)
            i = 0
            last_done = t0
            while len(lat) < n_q:
                now = time.monotonic_ns()
                while i < n_q and sched[i] <= now:
                    waiting[int(which[i])].append(i)
                    i += 1
                for gi in range(len(graphs)):
                    # a query without a free output slot of its graph waits (its latency still
                    # counts from its scheduled arrival); other graphs' queries go ahead
                    while waiting[gi] and free[gi]:
                        j = waiting[gi].popleft()
                        slot = free[gi].pop()
                        t = dobfs.dobfs_serve_submit(srv, gids[gi], int(pools[gi][ridx[j]]), slots[gi][slot])
                        inflight[t] = (gi, slot, int(sched[j]))
                done = dobfs.dobfs_serve_collect(srv, col)
                for t, r in done:
                    gi, slot, sc_ns = inflight.pop(t)
                    free[gi].append(slot)
                    lat.append((r.done_ns - sc_ns) * 1e-6)
                    last_done = max(last_done, r.done_ns)
                if not done and (i >= n_q or sched[i] > time.monotonic_ns()):
                    time.sleep(0.00005)
            lat = np.asarray(lat)
            span = (last_done - int(sched[0])) * 1e-9
            res["rates"][str(rate)] = {"queries": n_q, "p50_ms": float(np.percentile(lat, 50)),
                                       "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                                       "achieved_qps": n_q / span, "span_s": span,
                                       "vs_one_at_a_time": (n_q / span) / one_at_a_time_qps,
                                       "_latencies_ms": lat.tolist()}
            st1 = dobfs.dobfs_serve_get_stats(srv)
            coh = st1.cohorts - st0.cohorts
            res["rates"][str(rate)]["server"] = {
                "cohorts": int(coh), "mean_cohort_lanes": (st1.lanes_admitted - st0.lanes_admitted) / max(1, coh),
                "group_steps": int(st1.group_steps - st0.group_steps),
                "single_source_queries": int(st1.single_source - st0.single_source)}
        st = dobfs.dobfs_serve_get_stats(srv)
        res["server"] = {"lane_groups_created": int(st.groups_created), "iterations": int(st.iterations),
                         "cohorts": int(st.cohorts), "lanes_admitted": int(st.lanes_admitted),
                         "mean_cohort_lanes": st.lanes_admitted / max(1, st.cohorts),
                         "group_steps": int(st.group_steps), "single_source_queries": int(st.single_source)}
    finally:
        dobfs.dobfs_serve_destroy(srv)
        for g in graphs:
            g.close()
        del slots
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return res


def run_reference(args) -> None:
    """The reference arm: the CPU oracle, as it stands, on the bench's
    workload. Each step is the oracle's serial FIFO BFS (levels, one core)
    from one seeded root: in full on graphs of at most 2 * REF_STEP_ENTRIES
    stored entries, else stopped after REF_STEP_ENTRIES adjacency entries (a
    bounded sample of that root's BFS; TEPS = entries read / 2 / time)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import dobfs_inputs as inputs
    import oracle

    workload = args.workload or DEFAULT_WORKLOAD
    kind, size, _, _ = WORKLOADS[workload]
    info = host_info()
    osize = pick_oracle_size(kind, size, info["mem_available_gb"])
    t0 = time.perf_counter()
    spec, g = oracle_graph(inputs, oracle, kind, osize, info["cores"] or 1)
    build_s = time.perf_counter() - t0
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), g.n, args.steps + args.warmup, g.degrees() > 0)
    limit = None if g.nnz <= 2 * REF_STEP_ENTRIES else REF_STEP_ENTRIES
    oracle_timing(oracle, g, roots[:args.warmup], limit)
    hm, t_sum, _ = oracle_timing(oracle, g, roots[args.warmup:], limit)
    what = "full BFS" if limit is None else "BFS stopped after %d adjacency entries (of %d stored)" % (limit, g.nnz)
    sample = ("oracle serial FIFO BFS (levels, one core) on %s, one seeded root per step, %s; graph built by the "
              "oracle's threaded builder in %.0f s (not timed)" % (workload_name(kind, osize), what, build_s))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": hm, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_sum / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name(kind, osize), "scale": osize, "edgefactor": 16,
                   "generator": kind},
        "cpu_baseline": {"value": hm, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample,
                         "host": info},
        "e2e": {"value": hm, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def write_root_log(path: str, workload: str, rank: int, roots, ms, teps, levels, alg_bytes, peak: float,
                   options: str) -> None:
    """One JSON line per timed root: device time, TEPS, levels, algorithmic
    bytes, and the whole-BFS fraction of the HBM peak they imply."""
    with open(path, "w") as f:
        for r, t, e, lv, b in zip(roots, ms, teps, levels, alg_bytes):
            gbs = b / (t * 1e-3) / 1e9
            f.write(json.dumps({"workload": workload, "rank": rank, "root": int(r), "device_ms": t,
                                "gteps": e / (t * 1e-3) / 1e9, "teps_edges": int(e), "levels": int(lv),
                                "alg_bytes": int(b), "alg_gbs": gbs, "roofline_frac": gbs / peak,
                                "options": options}) + "\n")


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help="graph to time (default rmat28, the headline)")
    ap.add_argument("--scale", type=int, default=None, help="R-MAT scale other than the named workloads'")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-reindex", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--cpu-full", action="store_true",
                    help="CPU baseline: full oracle BFS from each root even on graphs where it samples")
    ap.add_argument("--cpu-roots", type=int, default=4, help="roots of the CPU baseline")
    ap.add_argument("--cpu-all-cores", action="store_true",
                    help="CPU baseline: also roots/s of full BFS, one per core on every core")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--batch-scale", type=int, default=24)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-BFS measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="arrival window per rate")
    ap.add_argument("--tune", action="store_true", help="tune the run options on 8 other roots first")
    ap.add_argument("--jsonl", default=None,
                    help="also write one JSON line per timed root to this file (rank r > 0: file.r)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.scale is not None and args.workload is None:
        key = "rmat%d" % args.scale
        if key not in WORKLOADS:
            WORKLOADS[key] = ("rmat", args.scale, ("REINDEX",), 64)
        args.workload = key
    if args.workload is None:
        args.workload = DEFAULT_WORKLOAD

    if args.impl == "reference":
        run_reference(args)
        return

    import torch

    import dobfs_inputs as inputs
    from paper_1503_04359_b300 import build as build_mod
    from paper_1503_04359_b300 import dobfs

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    if rank == 0:
        build_mod.build()
    if dist:
        dist.barrier()
    dobfs.load()
    dobfs.use_torch_allocator()
    dev = torch.cuda.current_device()

    kind, size, flag_names, _ = WORKLOADS[args.workload]
    spec = make_spec(inputs, kind, size)
    flags = 0
    for nm in flag_names:
        if nm and not (args.no_reindex and nm == "REINDEX"):
            flags |= getattr(dobfs, "DOBFS_GRAPH_" + nm)
    t0 = time.perf_counter()
    if kind == "rmat":
        g = dobfs.rmat_graph(spec, flags=flags)
    else:
        g = dobfs.chunglu_graph(spec, inputs.chunglu_cdf(spec), flags=flags)
    build_s = time.perf_counter() - t0
    info = g.info
    n = int(info.n_vertices)
    deg = g.degrees()
    roots_all = inputs.sample_roots(inputs.root_seed(spec.seed) + rank * 0x1000, n, args.steps + args.warmup, deg > 0)
    warm, roots = roots_all[:args.warmup], roots_all[args.warmup:]

    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    opts = dobfs.make_opts(stream=stream)
    tuning = None
    if args.tune:
        from paper_1503_04359_b300 import autotune
        tune_roots = inputs.sample_roots(inputs.root_seed(spec.seed) ^ 0x7E57, n, 8, deg > 0)
        t0 = time.perf_counter()
        _, rec = autotune.tune(g, tune_roots)
        opts = dobfs.make_opts(stream=stream, **rec["params"])
        tuning = {"policy": rec["policy"], "params": rec["params"], "sample_roots": len(tune_roots),
                  "default_ms_per_root": rec["default_ms"], "tuned_ms_per_root": rec["ms"],
                  "seconds": round(time.perf_counter() - t0, 1)}

    # untimed pass: per-root edge counts, levels and algorithmic bytes
    teps, alg_bytes, launches, levels = [], [], [], []
    for r in list(warm) + list(roots):
        st = g.run(int(r), level, parent, opts, want_stats=True)
        tr = g.trace()
        teps.append(st.teps_edges)
        alg_bytes.append(st.alg_bytes)
        levels.append(st.levels)
        # kernels: init + output + per level (switch + 2 expand kernels, + 1 conversion on a direction
        # change) + the closing switch
        k = 3
        prev = 0
        for t in tr:
            k += 3 + (1 if t.direction != prev else 0)
            prev = t.direction
        launches.append(k)
    teps, alg_bytes = teps[args.warmup:], alg_bytes[args.warmup:]
    launches, levels = launches[args.warmup:], levels[args.warmup:]

    # timed pass
    for r in warm:
        g.run(int(r), level, parent, opts)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(roots) + 1)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_bus_id(torch, dev)) as clk:
        wall0 = time.perf_counter()
        ev[0].record(stream)
        for i, r in enumerate(roots):
            g.run(int(r), level, parent, opts)
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(len(roots))]
    total_ms = sum(ms)
    rates = [e / (t * 1e-3) / 1e9 for e, t in zip(teps, ms)]
    hmean = len(rates) / sum(1.0 / x for x in rates)
    total_edges = float(sum(teps))
    clocks = clk.summary()

    # job value over ranks: all ranks' edges over the slowest rank's time
    job_value, job_ms = hmean, total_ms
    if dist:
        job_value, job_ms = aggregate_ranks(dist, "cuda", total_ms, total_edges)

    peak, peak_kind = _peaks()
    workload = workload_name(kind, size)
    if args.jsonl:
        write_root_log(args.jsonl if rank == 0 else "%s.%d" % (args.jsonl, rank), workload, rank, roots, ms, teps,
                       levels, alg_bytes, peak, "tuned" if tuning is not None else "defaults")

    # roofline of the dominant kernel: per-level events in host-driven mode on
    # a fixed root sample with the default options
    hl = dobfs.make_opts(stream=stream, flags=dobfs.DOBFS_RUN_HOST_LOOP)
    per_kind = {0: [0.0, 0], 1: [0.0, 0], 2: [0.0, 0]}  # direction (top-down, bottom-up, mixed) -> [ms, bytes]
    n_launch = {0: 0, 1: 0, 2: 0}
    roof_roots = inputs.sample_roots(inputs.root_seed(spec.seed) ^ 0x500F, n, 16, deg > 0)
    for r in roof_roots:
        g.run(int(r), level, parent, hl)
        torch.cuda.synchronize()
        for t in g.trace():
            per_kind[t.direction][0] += t.ms_main
            per_kind[t.direction][1] += t.alg_bytes
            n_launch[t.direction] += 1
    dom = max(per_kind, key=lambda k: per_kind[k][0])
    dom_ms, dom_bytes = per_kind[dom]
    achieved = (dom_bytes / n_launch[dom]) / ((dom_ms / n_launch[dom]) * 1e-3) / 1e9 if n_launch[dom] else 0.0
    step_ms = max(1e-9, sum(v[0] for v in per_kind.values()))
    by_step = {}
    for k, (k_ms, k_bytes) in per_kind.items():
        if not n_launch[k]:
            continue
        gbs = k_bytes / (k_ms * 1e-3) / 1e9
        by_step[STEP_NAMES[k]] = {"levels": n_launch[k], "time_share": k_ms / step_ms,
                                  "alg_bytes_per_level": k_bytes / n_launch[k], "achieved": gbs, "frac": gbs / peak}
    whole_gbs = (sum(alg_bytes) / (total_ms * 1e-3)) / 1e9
    # the same whole-BFS bytes with the output pass counted as 8 bytes per reached
    # vertex (its level and parent), without the writes of unreached vertices'
    # -1 entries and the map reads
    out_extra = 8 * n + (4 * n if info.reindexed else 0)
    whole_gbs_8r = (sum(b - out_extra for b in alg_bytes) / (total_ms * 1e-3)) / 1e9

    energy = energy_pass(torch, g, roots, level, parent, opts, teps, gpu_bus_id(torch, dev)) if rank == 0 else None

    # end to end through the C ABI with pinned host outputs (D2H inside the timed region)
    hl_lv = torch.empty(n, dtype=torch.int32, pin_memory=True)
    hl_pa = torch.empty(n, dtype=torch.int32, pin_memory=True)
    e2e_roots = roots[:max(1, min(args.e2e_steps, len(roots)))]
    g.run(int(e2e_roots[0]), hl_lv.numpy(), hl_pa.numpy(), opts)
    e2e_rates = []
    e2e_t = 0.0
    for i, r in enumerate(e2e_roots):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.run(int(r), hl_lv.numpy(), hl_pa.numpy(), opts)  # returns after the D2H copies completed
        dt = time.perf_counter() - t0
        e2e_t += dt
        e2e_rates.append(teps[i] / dt / 1e9)
    e2e_hm = len(e2e_rates) / sum(1.0 / x for x in e2e_rates)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.workload, n_roots=args.cpu_roots, full=args.cpu_full,
                           all_cores=args.cpu_all_cores)

    # the remaining measurements use their own graphs
    del level, parent, hl_lv, hl_pa
    g.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    batch = None
    default_wl = args.workload == DEFAULT_WORKLOAD
    # batched and served BFS shard as replicas: every rank runs its own on its
    # own GPU and graph copy; rank 0 combines (roots and queries over all ranks,
    # the slowest rank's time)
    if not args.no_batch and default_wl:
        batch = measure_batch(torch, inputs, dobfs, args.batch_scale, peak, rank=rank)
        if dist:
            allb = [None] * ws
            dist.all_gather_object(allb, batch)
            batch = combine_batch(allb)
    serve = None
    if not args.no_serve and default_wl:
        serve = measure_serve(torch, inputs, dobfs, seconds=args.serve_seconds, rank=rank)
        if dist:
            alls = [None] * ws
            dist.all_gather_object(alls, serve)
            serve = combine_serve(alls)
        serve = strip_private(serve)

    if rank != 0:
        return
    prof = profiled_traffic() if dom == 1 else None
    traffic = None
    if prof:  # DRAM bytes per algorithmic byte of the captured bottom-up levels, scaled to these levels
        traffic = prof["dram_bytes"] / prof["alg_bytes"] * (dom_bytes / n_launch[dom])
    result = {
        "metric": METRIC,
        "value": job_value,
        "unit": "GTEPS",
        "n_gpus": ws,
        "steps": len(roots),
        "warmup": args.warmup,
        "ms_per_step": job_ms / len(roots),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "config": {
            "workload": workload, "generator": kind,
            "scale": size, "seed": spec.seed,
            "n_vertices": n, "n_entries": int(info.n_entries), "n_nonisolated": int(info.n_nonisolated),
            "offsets_int64": int(info.offsets_int64), "reindexed": int(info.reindexed),
            "roots": len(roots), "parallelism": "replicas" if ws > 1 else "single-gpu",
            "l2": "inputs larger than L2 (graph %.1f GB resident), no flush" % (info.device_bytes / 1e9),
            "build_s": round(build_s, 2), "device_bytes": int(info.device_bytes),
            "run_options": "tuned" if tuning is not None else "defaults",
        },
        "per_root": {"ms_mean": total_ms / len(roots), "ms_min": min(ms), "ms_max": max(ms),
                     "gteps_min": min(rates), "gteps_max": max(rates), "levels_mean": float(np.mean(levels)),
                     "teps_edges_mean": total_edges / len(roots), "aggregate_gteps": total_edges / total_ms / 1e6,
                     "wall_s": wall},
        "roofline": {
            "kernel": STEP_KERNELS[dom],
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": peak_kind, "traffic": traffic,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the bottom-up levels of %s "
                               "(%s), per algorithmic byte, times this workload's algorithmic bytes per level"
                               % (prof["workload"], TRAFFIC_PROFILE)) if traffic is not None else None,
            "alg_bytes_per_level": (dom_bytes / n_launch[dom]) if n_launch[dom] else None,
            "levels_timed": n_launch[dom], "roots": len(roof_roots), "options": "defaults, host-driven levels",
            "by_step": by_step,
            "whole_bfs_alg_gbs": whole_gbs, "whole_bfs_frac": whole_gbs / peak,
            "whole_bfs_frac_out8r": whole_gbs_8r / peak,
            "whole_bfs_note": ("whole_bfs_frac counts the output pass as 8 n (level and parent of every vertex "
                               "written) + 4 n (map read, renumbered graphs) + 8 per reached vertex (its entry "
                               "gathered); whole_bfs_frac_out8r counts only 8 per reached vertex"),
            "alg_bytes_per_root": float(np.mean(alg_bytes)),
        },
        "e2e": {"value": e2e_hm, "unit": "GTEPS", "h2d_bytes_per_step": 4, "d2h_bytes_per_step": 8 * n,
                "steps": len(e2e_roots),
                "note": "dobfs_run with pinned host outputs; the step's input is the 4-byte root, passed by value"},
        "gpu_launches": int(sum(launches)),
        "clocks": clocks,
    }
    if tuning is not None:
        result["tuning"] = tuning
    if energy is not None:
        result["energy"] = energy
    if cpu is not None:
        result["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample", "host",
                                                      "same_workload", "oracle_build_s", "per_root_gteps")}
        if "all_cores" in cpu:
            result["cpu_baseline"]["all_cores"] = cpu["all_cores"]
    if batch is not None:
        result["batch"] = batch
    if serve is not None:
        result["serve"] = serve
    print(json.dumps(result))


if __name__ == "__main__":
    main()
