"""Pins for the CPU oracle (runs without a GPU).

The paper prints no worked example with values, so the oracle is pinned to
mathematics instead: brute-force matrix-power reachability on every root of
random tiny graphs, closed forms of textbook graph families, hand-worked
fixtures under tests/golden/, and planted mistakes that the invariant checker
must catch.
"""
import itertools
import os

import numpy as np
import pytest

import dobfs_inputs as inputs
import oracle
from oracle import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _graph(n, pairs):
    src = np.array([p[0] for p in pairs], dtype=np.int32)
    dst = np.array([p[1] for p in pairs], dtype=np.int32)
    return src, dst, oracle.csr_from_pairs(n, src, dst)


def _load_golden(name):
    n, pairs, exp = None, [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "n":
                n = int(vals[0])
            elif key == "e":
                pairs.append((int(vals[0]), int(vals[1])))
            else:
                exp[key] = [int(v) for v in vals]
    return n, pairs, exp


@pytest.mark.parametrize("name", ["petersen.txt", "two_triangles_and_isolated.txt"])
def test_golden_fixtures(name):
    n, pairs, exp = _load_golden(name)
    _, _, g = _graph(n, pairs)
    root = exp["root"][0]
    level, parent, _ = oracle.bfs(g, root)
    assert level.tolist() == exp["level"]
    assert parent.tolist() == exp["parent"]
    if "teps_edges" in exp:
        assert oracle.teps_edges(g, level) == exp["teps_edges"][0]
    assert oracle.check_bfs(g, root, level, parent)[0] == 0


def test_petersen_distance_distribution():
    # distance-regular with intersection array {3,2;1,1}: 1 / 3 / 6 per distance from every root
    n, pairs, _ = _load_golden("petersen.txt")
    _, _, g = _graph(n, pairs)
    for r in range(n):
        level, _, nlev = oracle.bfs(g, r)
        assert nlev == 3
        assert np.bincount(level).tolist() == [1, 3, 6]


def _random_pairs(rng, n, m):
    return [(int(rng.integers(n)), int(rng.integers(n))) for _ in range(m)]


@pytest.mark.parametrize("seed", range(12))
def test_oracle_matches_brute_force_all_roots(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 48))
    m = int(rng.integers(0, 3 * n + 1))
    pairs = _random_pairs(rng, n, m)
    src, dst, g = _graph(n, pairs)
    bl = brute.brute_levels(n, src, dst)
    for r in range(n):
        level, parent, _ = oracle.bfs(g, r)
        np.testing.assert_array_equal(level, bl[r])
        np.testing.assert_array_equal(parent, brute.brute_canonical_parent(n, src, dst, bl[r], r))
        assert oracle.check_bfs(g, r, level, parent)[0] == 0


def test_csr_matches_set_construction():
    rng = np.random.default_rng(7)
    for _ in range(20):
        n = int(rng.integers(1, 60))
        pairs = _random_pairs(rng, n, int(rng.integers(0, 200)))
        src, dst, g = _graph(n, pairs)
        nbrs = [set() for _ in range(n)]
        for u, v in pairs:
            if u != v:
                nbrs[u].add(v)
                nbrs[v].add(u)
        assert g.nnz == sum(len(s) for s in nbrs)
        for u in range(n):
            assert g.row(u).tolist() == sorted(nbrs[u])


def test_csr_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.csr_from_pairs(3, [0], [3])


# ----------------------------------------------------------------- closed forms
def _path(n):
    return [(i, i + 1) for i in range(n - 1)]


def test_path():
    n = 37
    _, _, g = _graph(n, _path(n))
    level, parent, nlev = oracle.bfs(g, 0)
    assert level.tolist() == list(range(n)) and nlev == n
    assert parent.tolist() == [0] + list(range(n - 1))
    level, _, _ = oracle.bfs(g, 10)
    assert level.tolist() == [abs(i - 10) for i in range(n)]


@pytest.mark.parametrize("n", [3, 4, 9, 10])
def test_cycle(n):
    _, _, g = _graph(n, _path(n) + [(n - 1, 0)])
    level, _, _ = oracle.bfs(g, 0)
    assert level.tolist() == [min(i, n - i) for i in range(n)]


def test_star():
    n = 17
    _, _, g = _graph(n, [(0, i) for i in range(1, n)])
    level, parent, _ = oracle.bfs(g, 0)
    assert level.tolist() == [0] + [1] * (n - 1)
    level, parent, _ = oracle.bfs(g, 5)
    assert level.tolist() == [1] + [2] * 4 + [0] + [2] * (n - 6)
    assert parent[1] == 0 and parent[0] == 5


def test_complete():
    n = 12
    _, _, g = _graph(n, list(itertools.combinations(range(n), 2)))
    for r in (0, 7):
        level, parent, _ = oracle.bfs(g, r)
        assert level.tolist() == [0 if i == r else 1 for i in range(n)]
        assert all(parent[i] == r for i in range(n))


def test_binary_tree_heap_order():
    n = 63
    _, _, g = _graph(n, [((i - 1) // 2, i) for i in range(1, n)])
    level, parent, _ = oracle.bfs(g, 0)
    assert level.tolist() == [int(np.floor(np.log2(i + 1))) for i in range(n)]
    assert parent.tolist() == [0] + [(i - 1) // 2 for i in range(1, n)]


def test_grid_manhattan():
    r, c = 7, 9
    idx = lambda i, j: i * c + j  # noqa: E731
    pairs = [(idx(i, j), idx(i, j + 1)) for i in range(r) for j in range(c - 1)]
    pairs += [(idx(i, j), idx(i + 1, j)) for i in range(r - 1) for j in range(c)]
    _, _, g = _graph(r * c, pairs)
    level, _, _ = oracle.bfs(g, idx(2, 3))
    assert level.tolist() == [abs(i - 2) + abs(j - 3) for i in range(r) for j in range(c)]


def test_disjoint_union_and_isolated_root():
    # path 0..4 and cycle 5..9, vertex 10 isolated
    pairs = _path(5) + [(5 + i, 5 + (i + 1) % 5) for i in range(5)]
    _, _, g = _graph(11, pairs)
    level, parent, _ = oracle.bfs(g, 0)
    assert level.tolist() == [0, 1, 2, 3, 4] + [-1] * 6
    assert parent[5:].tolist() == [-1] * 6
    level, parent, nlev = oracle.bfs(g, 10)
    assert level.tolist() == [-1] * 10 + [0] and nlev == 1
    assert parent.tolist() == [-1] * 10 + [10]
    assert oracle.teps_edges(g, level) == 0


def test_components_equal_brute_reachability():
    rng = np.random.default_rng(3)
    for _ in range(10):
        n = int(rng.integers(1, 40))
        pairs = _random_pairs(rng, n, int(rng.integers(0, n + 5)))
        src, dst, g = _graph(n, pairs)
        bl = brute.brute_levels(n, src, dst)
        comp = oracle.components(g)
        for u in range(n):
            for v in range(n):
                assert (comp[u] == comp[v]) == (bl[u, v] >= 0)
            assert comp[u] == min(v for v in range(n) if bl[u, v] >= 0)


def test_teps_edges_counts_component_edges():
    rng = np.random.default_rng(5)
    for _ in range(10):
        n = int(rng.integers(2, 40))
        pairs = _random_pairs(rng, n, int(rng.integers(0, 3 * n)))
        src, dst, g = _graph(n, pairs)
        r = int(rng.integers(n))
        level, _, _ = oracle.bfs(g, r)
        und = {frozenset((u, v)) for u, v in pairs if u != v and level[u] >= 0}
        assert oracle.teps_edges(g, level) == len(und)


# ----------------------------------------------------------------- planted mistakes
def _rmat_small():
    spec = inputs.rmat(10)
    g = oracle.csr_from_rmat(spec)
    deg = g.degrees()
    root = int(inputs.sample_roots(inputs.root_seed(spec.seed), g.n, 1, deg > 0)[0])
    return spec, g, root


def _liftable(g, level):
    for v in np.flatnonzero(level >= 2).tolist():
        if all(level[u] in (level[v] - 1, level[v]) for u in g.row(v).tolist()):
            return v
    raise AssertionError("no liftable vertex")


def test_checker_catches_planted_mistakes():
    spec, g, root = _rmat_small()
    level, parent, _ = oracle.bfs(g, root)
    assert oracle.check_bfs(g, root, level, parent)[0] == 0
    reached = np.flatnonzero(level > 1)
    v = int(reached[0])

    bad = level.copy(); bad[root] = 1
    assert oracle.check_bfs(g, root, bad, parent)[0] == 1
    badp = parent.copy(); badp[root] = -1
    assert oracle.check_bfs(g, root, level, badp)[0] == 2
    bad = level.copy(); bad[v] += 2           # edge spans > 1 level
    assert oracle.check_bfs(g, root, bad, None)[0] in (3, 10)
    bad = level.copy(); bad[v] = -1          # drop a reached vertex
    assert oracle.check_bfs(g, root, bad, None)[0] == 4
    badp = parent.copy()                      # parent that is not a neighbour
    non_nbr = next(u for u in range(g.n) if u != v and u not in set(g.row(v).tolist()))
    badp[v] = non_nbr
    assert oracle.check_bfs(g, root, level, badp)[0] == 5
    same = [u for u in g.row(v).tolist() if level[u] == level[v]]
    if same:                                  # neighbour on the same level
        badp = parent.copy(); badp[v] = same[0]
        assert oracle.check_bfs(g, root, level, badp)[0] == 6
    # a vertex lifted one level whose neighbours all sit on its level or one
    # up keeps every edge within one level but loses its neighbour one level up
    bad = level.copy(); bad[_liftable(g, level)] -= 1
    assert oracle.check_bfs(g, root, bad, None)[0] == 10
    _, _, g3 = _graph(3, _path(3))
    assert oracle.check_bfs(g3, 0, np.array([0, 1, 1], dtype=np.int32), None)[0] == 10
    un = np.flatnonzero(level < 0)
    if len(un):
        badp = parent.copy(); badp[int(un[0])] = root
        assert oracle.check_bfs(g, root, level, badp)[0] == 7


def test_stream_check_matches_csr_check():
    spec, g, root = _rmat_small()
    level, parent, _ = oracle.bfs(g, root)
    rc, _, canon, has_nbr = oracle.check_bfs_rmat_stream(spec, root, level, parent, want_canon=True,
                                                         want_has_nbr=True)
    assert rc == 0
    np.testing.assert_array_equal(canon, parent)
    np.testing.assert_array_equal(has_nbr.astype(bool), g.degrees() > 0)
    v = int(np.flatnonzero(level > 1)[0])
    bad = level.copy(); bad[v] = -1
    assert oracle.check_bfs_rmat_stream(spec, root, bad, None)[0] == 4
    bad = level.copy(); bad[level > 0] += 1
    assert oracle.check_bfs_rmat_stream(spec, root, bad, None)[0] == 3
    bad = level.copy(); bad[_liftable(g, level)] -= 1
    assert oracle.check_bfs_rmat_stream(spec, root, bad, None)[0] == 10
    badp = parent.copy()
    non_nbr = next(u for u in range(g.n) if u != v and u not in set(g.row(v).tolist()) and level[u] == level[v] - 1)
    badp[v] = non_nbr
    assert oracle.check_bfs_rmat_stream(spec, root, level, badp)[0] == 9


def test_csr_from_rmat_equals_pairs_path():
    spec = inputs.rmat(9, edgefactor=8)
    a = oracle.csr_from_rmat(spec)
    src, dst = inputs.rmat_pairs(spec)
    b = oracle.csr_from_pairs(spec.n_vertices, src, dst)
    np.testing.assert_array_equal(a.off, b.off)
    np.testing.assert_array_equal(a.cols, b.cols)


def test_bfs_many_equals_single():
    spec, g, root = _rmat_small()
    roots = inputs.sample_roots(123, g.n, 5, g.degrees() > 0)
    lv, pa = oracle.bfs_many(g, roots)
    for i, r in enumerate(roots):
        l1, p1, _ = oracle.bfs(g, int(r))
        np.testing.assert_array_equal(lv[i], l1)
        np.testing.assert_array_equal(pa[i], p1)


def test_stream_multi_equals_single_and_isolates_roots():
    spec, g, root = _rmat_small()
    roots = inputs.sample_roots(77, g.n, 3, g.degrees() > 0)
    lv, pa = oracle.bfs_many(g, roots)
    rc, bad, canon = oracle.check_bfs_rmat_stream_multi(spec, roots, lv, pa, want_canon=True)
    assert rc.tolist() == [0, 0, 0]
    np.testing.assert_array_equal(canon, pa)
    # a planted mistake in root 1 only fails root 1
    lv2 = lv.copy()
    v = int(np.flatnonzero(lv2[1] > 1)[0])
    lv2[1, v] = -1
    rc, bad, _ = oracle.check_bfs_rmat_stream_multi(spec, roots, lv2, pa)
    assert rc.tolist() == [0, 4, 0]
    # the same check over the pairs held in arrays
    src, dst = inputs.rmat_pairs(spec)
    rc, bad, canon2, has_nbr = oracle.check_bfs_pairs_multi(g.n, src, dst, roots, lv, pa, want_canon=True,
                                                            want_has_nbr=True)
    assert rc.tolist() == [0, 0, 0]
    np.testing.assert_array_equal(canon2, pa)
    np.testing.assert_array_equal(has_nbr.astype(bool), g.degrees() > 0)
    badp = pa.copy()
    badp[2, int(np.flatnonzero(lv[2] > 0)[0])] = -5
    rc, _, _, _ = oracle.check_bfs_pairs_multi(g.n, src, dst, roots, lv, badp)
    assert rc.tolist() == [0, 0, 5]


def test_csr_from_rmat_par_equals_serial_and_pairs():
    """The threaded build places entries in another order inside each row;
    after the row sort it must give the serial CSR (itself pinned to the
    set-based construction through csr_from_pairs) at any thread count."""
    for scale, ef in ((9, 8), (12, 16), (15, 16)):
        spec = inputs.rmat(scale, edgefactor=ef)
        a = oracle.csr_from_rmat(spec)
        src, dst = inputs.rmat_pairs(spec)
        b = oracle.csr_from_pairs(spec.n_vertices, src, dst)
        for nt in (1, 3, 8):
            c = oracle.csr_from_rmat_par(spec, n_threads=nt)
            np.testing.assert_array_equal(c.off, a.off)
            np.testing.assert_array_equal(c.cols, a.cols)
        np.testing.assert_array_equal(a.off, b.off)
        np.testing.assert_array_equal(a.cols, b.cols)
        for nt in (1, 5):
            c = oracle.csr_from_pairs_par(spec.n_vertices, src, dst, n_threads=nt)
            np.testing.assert_array_equal(c.off, a.off)
            np.testing.assert_array_equal(c.cols, a.cols)


def test_csr_from_pairs_par_set_construction_and_range():
    rng = np.random.default_rng(11)
    for _ in range(10):
        n = int(rng.integers(1, 60))
        pairs = _random_pairs(rng, n, int(rng.integers(0, 200)))
        src, dst, g = _graph(n, pairs)
        c = oracle.csr_from_pairs_par(n, src, dst, n_threads=4)
        np.testing.assert_array_equal(c.off, g.off)
        np.testing.assert_array_equal(c.cols, g.cols)
    with pytest.raises(ValueError):
        oracle.csr_from_pairs_par(3, [0], [3])


def test_bfs_partial_path_closed_form():
    """Path 0-1-...-(n-1) from vertex 0: rows are read in queue order (degree
    1, then 2, 2, ...); after the rows of vertices 0..k, 1 + 2k entries have
    been read and vertices 0..k+1 carry their levels. The BFS stops at the
    first row boundary with at least max_entries entries read."""
    n = 41
    _, _, g = _graph(n, _path(n))
    for budget in range(1, 2 * n):
        level, read = oracle.bfs_partial(g, 0, budget)
        k = min(max(0, -(-(budget - 1) // 2)), n - 1)
        expect_read = 1 + 2 * k if k < n - 1 else 2 * (n - 1)
        reached = min(k + 2, n)
        assert read == expect_read, (budget, read, expect_read)
        assert level[:reached].tolist() == list(range(reached))
        assert (level[reached:] == -1).all()


def test_bfs_partial_prefix_of_full_bfs():
    spec, g, root = _rmat_small()
    full, _, _ = oracle.bfs(g, root, want_parent=False)
    total = int(g.degrees()[full >= 0].sum())
    lv, read = oracle.bfs_partial(g, root, g.nnz + 1)
    np.testing.assert_array_equal(lv, full)
    assert read == total
    maxdeg = int(g.degrees().max())
    for budget in (1, 10, 100, total // 7, total // 2, total - 1):
        lv, read = oracle.bfs_partial(g, root, budget)
        got = lv >= 0
        assert np.array_equal(lv[got], full[got])
        assert min(budget, total) <= read < budget + maxdeg


def test_stream_check_vertex_major_equals_root_major():
    """The vertex-major layout (entry (r, v) at v*R + r) changes only where
    the per-root arrays live: the same planted mistakes give the same rule,
    vertex and canonical parents as the root-major layout."""
    spec, g, root = _rmat_small()
    roots = inputs.sample_roots(91, g.n, 7, g.degrees() > 0)
    lv, pa = oracle.bfs_many(g, roots)
    lv, pa = lv.copy(), pa.copy()
    deep = [int(np.flatnonzero(lv[i] > 1)[0]) for i in range(7)]
    lv[1, deep[1]] = -1                                   # rule 4
    pa[2, deep[2]] = -5                                   # rule 5
    v = deep[3]                                           # rule 9: a non-neighbour one level up
    nb = set(g.row(v).tolist())
    pa[3, v] = next(u for u in range(g.n) if u != v and u not in nb and lv[3, u] == lv[3, v] - 1)
    v = deep[4]                                           # rule 6: a neighbour on the same level
    same = [u for u in g.row(v).tolist() if lv[4, u] == lv[4, v]]
    if same:
        pa[4, v] = same[0]
    lv[5, int(roots[5])] = 1                              # rule 1
    rm = oracle.check_bfs_rmat_stream_multi(spec, roots, lv, pa, want_canon=True)
    vm = oracle.check_bfs_rmat_stream_multi(spec, roots, np.ascontiguousarray(lv.T), np.ascontiguousarray(pa.T),
                                            want_canon=True, vertex_major=True)
    assert rm[0].tolist()[:4] == [0, 4, 5, 9] and rm[0][5] == 1
    np.testing.assert_array_equal(rm[0], vm[0])
    np.testing.assert_array_equal(rm[1], vm[1])
    np.testing.assert_array_equal(rm[2], vm[2].T)
    src, dst = inputs.rmat_pairs(spec)
    pm = oracle.check_bfs_pairs_multi(g.n, src, dst, roots, np.ascontiguousarray(lv.T), np.ascontiguousarray(pa.T),
                                      want_canon=True, vertex_major=True)
    np.testing.assert_array_equal(rm[0], pm[0])
    np.testing.assert_array_equal(rm[2], pm[2].T)
