"""Pins for the seeded input generators (runs without a GPU)."""
import math

import numpy as np
import pytest

import dobfs_inputs as inputs


def test_mix64_python_equals_c():
    lib = inputs._load()
    for z in [0, 1, 2, 0xDEADBEEF, (1 << 64) - 1, 0x5EED0000 + 28]:
        assert inputs.mix64(z) == lib.gen_c_mix64(z)
    # SplitMix64 seeded with 0: first outputs are the published sequence of the
    # reference generator (state advanced by the golden gamma before mixing)
    assert inputs.mix64(0) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 1000, 1 << 12, 5000])
def test_perm_is_bijection(n):
    img = sorted(inputs.perm(x, n, 99) for x in range(n))
    assert img == list(range(n))


def test_rmat_quadrant_frequencies():
    # per bit position, the source bit is 0 with probability A+B and the
    # destination bit is 0 with probability A+C; test at 5 binomial sigmas
    spec = inputs.RmatSpec(scale=16, edgefactor=4, seed=42)
    src, dst = inputs.rmat_pairs(spec, relabel=False)
    m = len(src)
    a, b, c = spec.a, spec.b, spec.c
    for bit in range(spec.scale):
        su = ((src >> bit) & 1) == 0
        sv = ((dst >> bit) & 1) == 0
        for obs, p in ((su.mean(), a + b), (sv.mean(), a + c), ((su & sv).mean(), a)):
            assert abs(obs - p) < 5 * math.sqrt(p * (1 - p) / m), (bit, obs, p)


def test_rmat_deterministic_and_seeded():
    s1 = inputs.rmat(12)
    a = inputs.rmat_pairs(s1, k0=100, count=1000)
    b = inputs.rmat_pairs(s1)
    np.testing.assert_array_equal(a[0], b[0][100:1100])
    np.testing.assert_array_equal(a[1], b[1][100:1100])
    c = inputs.rmat_pairs(inputs.rmat(12, seed=1))
    assert (c[0] != b[0]).mean() > 0.5
    assert b[0].min() >= 0 and b[0].max() < s1.n_vertices


def test_rmat_relabel_is_the_vertex_permutation():
    spec = inputs.rmat(11)
    raw = inputs.rmat_pairs(spec, relabel=False, count=500)
    rel = inputs.rmat_pairs(spec, count=500)
    for x, y in zip(raw[0][:50], rel[0][:50]):
        assert inputs.perm(int(x), spec.n_vertices, spec.seed) == int(y)


def test_rmat_thresholds():
    ta, tab, tabc = inputs.rmat_thresholds(0.57, 0.19, 0.19)
    assert ta == math.floor(0.57 * 2 ** 32)
    assert ta < tab < tabc < 2 ** 32
    assert abs((2 ** 32 - tabc) / 2 ** 32 - 0.05) < 1e-9


def test_chunglu_weights_and_draws():
    spec = inputs.chunglu(14, max_weight=float(1 << 10))
    cdf = inputs.chunglu_cdf(spec)
    w = np.diff(np.concatenate([[0], cdf.astype(np.float64)])) / float(1 << 20)
    assert abs(w.mean() - spec.mean_degree) < 1e-3 * spec.mean_degree
    assert np.all(np.diff(w) <= 1e-9)                     # non-increasing in the index
    assert 0.7 * 1024 < w[0] < 1.3 * 1024                  # max weight near the target
    # power law: w_i ~ (i+i0)^(-1/(gamma-1)) -> log-log slope over the tail
    i = np.array([1000, 8000])
    slope = np.log(w[i[1]] / w[i[0]]) / np.log(i[1] / i[0])
    assert abs(slope + 1 / (spec.gamma - 1)) < 0.05
    src, dst = inputs.chunglu_pairs(spec, cdf)
    assert len(src) == spec.n_pairs
    # draw frequency of the heaviest vertex matches its weight share (5 sigma)
    heavy = inputs.perm(0, spec.n_vertices, spec.seed)
    hits = int((src == heavy).sum() + (dst == heavy).sum())
    p = w[0] / w.sum()
    draws = 2 * len(src)
    assert abs(hits - p * draws) < 5 * math.sqrt(draws * p * (1 - p))


def test_sample_roots():
    deg = np.zeros(1000, dtype=np.int64)
    deg[::3] = 1
    r = inputs.sample_roots(5, 1000, 50, deg > 0)
    assert len(set(r.tolist())) == 50
    assert np.all(deg[r] > 0)
    np.testing.assert_array_equal(r, inputs.sample_roots(5, 1000, 50, deg > 0))
    with pytest.raises(ValueError):
        inputs.sample_roots(5, 10, 5, np.zeros(10, dtype=bool))


def test_chunglu_bucketed_search_equals_plain_search():
    spec = inputs.chunglu(16, max_weight=float(1 << 12))
    cdf = inputs.chunglu_cdf(spec)
    a = inputs.chunglu_pairs(spec, cdf, count=200_000)
    b = inputs.chunglu_pairs(spec, cdf, count=200_000, plain_search=True)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
