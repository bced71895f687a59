"""Autotuner: the coordinate-descent search and the cache on the host, and
on the GPU that tuned options keep the levels bit-exact (tuning changes only
the speed)."""
import numpy as np
import pytest

import dobfs_inputs as inputs
import oracle

torch = pytest.importorskip("torch")


def _autotune():
    from paper_1503_04359_b300 import autotune
    return autotune


def test_descend_finds_separable_minimum():
    at = _autotune()
    grid = {"a": [1, 2, 4, 8, 16], "b": [0, 1, 2, 3]}
    calls = []

    def cost(p):
        calls.append(dict(p))
        return 10.0 + (np.log2(p["a"]) - 3) ** 2 + 0.5 * (p["b"] - 1) ** 2

    best, ms, log = at.descend(grid, cost, {"a": 1, "b": 3})
    assert best == {"a": 8, "b": 1} and ms == pytest.approx(10.0)
    # every evaluation is logged once; no point is measured twice
    keys = [tuple(sorted(c.items())) for c in calls]
    assert len(keys) == len(set(keys)) == len(log)


def test_descend_keeps_start_within_min_gain():
    at = _autotune()
    grid = {"a": [1, 2, 3]}
    best, ms, _ = at.descend(grid, lambda p: 100.0 - 0.1 * p["a"], {"a": 1}, min_gain=0.01)
    assert best == {"a": 1} and ms == 99.9  # 0.2 % faster is below the 1 % threshold


def test_cache_round_trip(tmp_path):
    at = _autotune()
    path = str(tmp_path / "sub" / "tuned.json")
    assert at.load_cache(path) == {}
    at.save_cache(path, "k1", {"params": {"alpha": 8}, "ms": 1.0})
    at.save_cache(path, "k2", {"params": {"beta": 48}, "ms": 2.0})
    c = at.load_cache(path)
    assert c["k1"]["params"] == {"alpha": 8} and c["k2"]["ms"] == 2.0


@pytest.mark.gpu
def test_tuned_options_keep_levels_exact(tmp_path):
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_04359_b300 import build, dobfs
    build.build()
    dobfs.load()
    dobfs.use_torch_allocator()
    at = _autotune()
    spec = inputs.rmat(14)
    og = oracle.csr_from_rmat(spec)
    g = dobfs.rmat_graph(spec)
    deg = og.degrees()
    tune_roots = inputs.sample_roots(inputs.root_seed(spec.seed) ^ 0x7E57, og.n, 4, deg > 0)
    path = str(tmp_path / "tuned.json")
    opts, rec = at.tune(g, tune_roots, cache_path=path)
    assert rec["policy"] in ("alpha_beta", "static") and rec["ms"] > 0 and rec["default_ms"] > 0
    assert set(rec["policies"]) == {"alpha_beta", "static"}
    assert rec["ms"] <= min(p["ms"] for p in rec["policies"].values())
    # a second call is served from the cache without timing anything
    saved = at._time_single
    at._time_single = None
    try:
        opts2, rec2 = at.tune(g, tune_roots, cache_path=path)
    finally:
        at._time_single = saved
    assert rec2["params"] == rec["params"]
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 6, deg > 0)
    ref, _ = oracle.bfs_many(og, roots, want_parent=False)
    lv = torch.empty(og.n, dtype=torch.int32, device="cuda")
    for k, r in enumerate(roots):
        g.run(int(r), lv, None, opts2)
        np.testing.assert_array_equal(lv.cpu().numpy(), ref[k])
    bopts, brec = at.tune_batch(g, roots)
    out = torch.empty((len(roots), og.n), dtype=torch.int32, device="cuda")
    dobfs.dobfs_run_batch(g.handle, torch.from_numpy(np.ascontiguousarray(roots, dtype=np.int32)).cuda(), out,
                          opts=bopts)
    np.testing.assert_array_equal(out.cpu().numpy(), np.stack(ref))
    g.close()
