"""Host logic of bench.py: the replica aggregation over ranks (gloo, two
processes on the CPU) and the lookup of committed ncu traffic."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, inputs, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    ms, edges = inputs[rank]
    q.put((rank, bench.aggregate_ranks(dist, "cpu", ms, edges)))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_ranks_gloo_two_processes():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    inputs = [(10.0, 1e9), (20.0, 3e9)]  # rank 1 is the slowest
    procs = [ctx.Process(target=_worker, args=(r, 2, port, inputs, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        value, mx = got[r]
        assert mx == 20.0
        assert value == pytest.approx(4e9 / 0.020 / 1e9)


def test_profiled_traffic_needs_matching_sources(tmp_path, monkeypatch):
    prof = tmp_path / "p.md"
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(prof))
    rec = {"kernel_sha256": bench.kernel_sha256(), "workload": "rmat-s24-ef16", "dram_bytes": 150, "alg_bytes": 100}
    prof.write_text("summary\n<!-- traffic %s -->\n" % json.dumps(rec))
    got = bench.profiled_traffic()
    assert got["dram_bytes"] / got["alg_bytes"] == 1.5 and got["workload"] == "rmat-s24-ef16"
    rec["kernel_sha256"] = "0" * 64
    prof.write_text("<!-- traffic %s -->" % json.dumps(rec))
    assert bench.profiled_traffic() is None
    prof.write_text("no record")
    assert bench.profiled_traffic() is None


def test_workload_names_and_oracle_memory():
    assert bench.workload_name("rmat", 28) == "rmat-s28-ef16"
    assert bench.workload_name("chunglu", 26).startswith("chunglu-2^26")
    # scale 28: 4.3 G pairs -> 34.4 GB of columns before de-duplication, plus offsets, cursors, outputs
    assert 38 < bench.oracle_host_gb("rmat", 28) < 42
    assert bench.pick_oracle_size("rmat", 28, None) == 28
    assert bench.pick_oracle_size("rmat", 28, 1000.0) == 28
    assert bench.pick_oracle_size("rmat", 28, 30.0) == 27
    assert set(bench.WORKLOADS) >= {"rmat16", "rmat22", "rmat28", "chunglu26"}


def test_cpu_baseline_small_workload(monkeypatch):
    """The oracle leg on a small R-MAT workload: full BFS (the graph is below
    the sampling threshold), 2 roots, host description recorded."""
    monkeypatch.setitem(bench.WORKLOADS, "rmat12", ("rmat", 12, ("REINDEX",), 8))
    out = bench.cpu_baseline("rmat12", n_roots=2, all_cores=True)
    assert out["value"] > 0 and out["cores"] == 1 and out["same_workload"]
    assert "rmat-s12-ef16" in out["sample"] and "full BFS" in out["sample"]
    assert out["host"]["cores"] >= 1 and out["all_cores"]["roots"] >= 1


def test_cpu_baseline_samples_large_graphs(monkeypatch):
    """Above 2 * CPU_SAMPLE_ENTRIES stored entries the oracle's BFS is stopped
    after CPU_SAMPLE_ENTRIES entries per root."""
    monkeypatch.setattr(bench, "CPU_SAMPLE_ENTRIES", 1 << 12)
    monkeypatch.setitem(bench.WORKLOADS, "rmat12", ("rmat", 12, ("REINDEX",), 8))
    out = bench.cpu_baseline("rmat12", n_roots=2)
    assert "stopped after 4096 adjacency entries" in out["sample"]


def test_ncu_summary_groups_bottom_up_levels(tmp_path):
    from paper_1503_04359_b300 import ncu_summary
    rows = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    seq = [("k_bu<long, 0>", 3.0), ("k_bu<long, 1>", 9.0), ("k_bu_long<long>", 1.0),  # a mixed level: left out
           ("k_bu<long, 0>", 100.0), ("k_bu_long<long>", 5.0),    # bottom-up level 1
           ("k_td_bin<long, 0>", 7.0),
           ("k_bu<long, 0>", 50.0), ("k_bu_long<long>", 0.0),     # level 2
           ("k_bu<long, 0>", 20.0), ("k_bu_long<long>", 2.0)]     # level 3
    for i, (name, mb) in enumerate(seq):
        rows.append('"%d","void dobfs::(anonymous namespace)::%s(args)","dram__bytes_read.sum","Mbyte","%s"' % (i, name, mb))
        rows.append('"%d","void dobfs::(anonymous namespace)::%s(args)","dram__bytes_write.sum","Kbyte","0"' % (i, name))
        rows.append('"%d","void dobfs::(anonymous namespace)::%s(args)","gpu__time_duration.sum","usecond","10"' % (i, name))
    p = tmp_path / "x.csv"
    p.write_text("==PROF== noise\n" + "\n".join(rows) + "\n")
    launches = ncu_summary.read_launches(str(p))
    assert len(launches) == len(seq)
    lv = ncu_summary.bu_levels(launches)
    assert [x["bytes"] for x in lv] == [105e6, 50e6, 22e6]
    assert [x["launches"] for x in lv] == [2, 2, 2]
    table = {k: (c, t) for k, c, t, _ in ncu_summary.launch_table(launches)}
    assert table["k_bu<long, 0>"] == (4, 40.0) and table["k_bu_long<long>"] == (4, 40.0)


def test_per_root_jsonl(tmp_path):
    p = tmp_path / "roots.jsonl"
    bench.write_root_log(str(p), "rmat-s10-ef16-reindex", 0, [5, 9], [2.0, 4.0], [4_000_000, 2_000_000], [6, 7],
                         [6_400_000_000, 3_200_000_000], 6400.0, "defaults")
    rows = [json.loads(x) for x in p.read_text().splitlines()]
    assert [r["root"] for r in rows] == [5, 9]
    assert rows[0]["gteps"] == pytest.approx(4e6 / 2e-3 / 1e9)
    assert rows[1]["levels"] == 7 and rows[1]["teps_edges"] == 2_000_000
    # 6.4e9 bytes in 2 ms = 3200 GB/s = half of the 6400 GB/s peak
    assert rows[0]["alg_gbs"] == pytest.approx(3200.0)
    assert rows[0]["roofline_frac"] == pytest.approx(0.5)
    assert all(r["workload"] == "rmat-s10-ef16-reindex" and r["options"] == "defaults" for r in rows)


def _fake_batch(rank):
    ms = 10.0 * (rank + 1)  # rank 1 is the slowest
    return {"workload": "rmat-s24-ef16", "sequential": {"roots": 64, "ms": 20.0 + rank, "roots_per_s": 0.0,
                                                        "gteps": 1.0},
            "batches": {"64": {"ms": ms, "roots_per_s": 0.0, "speedup_vs_sequential": 0.0, "gteps_est": 100.0,
                               "roofline": {"bound": "hbm", "alg_bytes": 1e9, "achieved": 0.0, "peak": 6000.0,
                                            "unit": "GB/s", "frac": 0.0}}}}


def _fake_serve(rank):
    lat = [1.0 + rank, 2.0 + rank, 3.0 + rank]
    return {"workload": "x", "one_at_a_time": {"qps": 1000.0, "mean_device_ms_per_graph": [1.0]},
            "rates": {"2000": {"queries": 3, "span_s": 0.5 + rank, "achieved_qps": 0.0, "p50_ms": 0.0,
                               "p99_ms": 0.0, "mean_ms": 0.0, "vs_one_at_a_time": 0.0, "server": {"cohorts": 1},
                               "_latencies_ms": lat}}}


def _legs_worker(rank, ws, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    allb, alls = [None] * ws, [None] * ws
    dist.all_gather_object(allb, _fake_batch(rank))
    dist.all_gather_object(alls, _fake_serve(rank))
    q.put((rank, bench.combine_batch(allb), bench.strip_private(bench.combine_serve(alls))))
    dist.barrier()
    dist.destroy_process_group()


def test_batch_and_serve_legs_combine_over_two_gloo_ranks():
    """Batched and served BFS run as replicas: roots and queries of all ranks
    over the slowest rank's time, latency percentiles over all queries."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_legs_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (b, s)) for r, b, s in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        b, s = got[r]
        x = b["batches"]["64"]
        assert x["ms"] == 20.0 and x["roots_per_s"] == pytest.approx(128 / 0.020)
        assert b["sequential"]["roots"] == 128 and b["sequential"]["ms"] == 21.0
        assert x["speedup_vs_sequential"] == pytest.approx((128 / 0.020) / (128 / 0.021))
        assert x["roofline"]["alg_bytes"] == 2e9 and x["roofline"]["peak"] == 12000.0
        assert x["roofline"]["frac"] == pytest.approx(2e9 / 0.020 / 1e9 / 12000.0)
        y = s["rates"]["2000"]
        assert y["queries"] == 6 and y["achieved_qps"] == pytest.approx(6 / 1.5)
        assert y["p50_ms"] == pytest.approx(2.5) and "_latencies_ms" not in y
        assert s["one_at_a_time"]["qps"] == 2000.0 and s["replicas"] == 2
