"""Graph files (dobfs_graph_save / dobfs_graph_load) through the C ABI.

- Round trip: the loaded graph has the saved CSR, map and statistics, and its
  BFS levels are bit-exact with the oracle's.
- The format itself is pinned by a writer written here from the layout the
  header documents: a file written from the oracle's CSR loads, and its BFS
  matches the oracle.
- Damaged files fail with DOBFS_ERR_IO (bad magic or version, truncation,
  trailing data, flipped payload bytes); files with a valid checksum whose
  CSR breaks an invariant of the build fail with DOBFS_ERR_BAD_GRAPH before
  any BFS kernel sees them.
"""
import struct

import numpy as np
import pytest

import dobfs_inputs as inputs
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MASK = (1 << 64) - 1
FNV_BASIS, FNV_PRIME = 0xCBF29CE484222325, 0x100000001B3


@pytest.fixture(scope="module")
def d():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_04359_b300 import build, dobfs
    build.build()
    dobfs.load()
    dobfs.use_torch_allocator()
    return dobfs


def _checksum(payload: bytes) -> int:
    """Four FNV-1a streams over the 64-bit words (word i -> stream i mod 4),
    folded by FNV-1a together with the word count."""
    words = np.frombuffer(payload, dtype="<u8")
    h = [FNV_BASIS] * 4
    for i, w in enumerate(words.tolist()):
        h[i & 3] = ((h[i & 3] ^ w) * FNV_PRIME) & MASK
    r = FNV_BASIS
    for x in h:
        r = ((r ^ x) * FNV_PRIME) & MASK
    return ((r ^ len(words)) * FNV_PRIME) & MASK


def _pad8(b: bytes) -> bytes:
    return b + bytes(-len(b) % 8)


def _write_file(path, off, cols, n2o=None, off64=True, version=1, magic=b"DOBFSCSR", checksum=None):
    n = len(off) - 1
    payload = _pad8(np.asarray(off, dtype="<i8" if off64 else "<i4").tobytes())
    payload += _pad8(np.asarray(cols, dtype="<i4").tobytes())
    if n2o is not None:
        payload += _pad8(np.asarray(n2o, dtype="<i4").tobytes())
    flags = (1 if off64 else 0) | (2 if n2o is not None else 0)
    ck = _checksum(payload) if checksum is None else checksum
    head = magic + struct.pack("<IIqqQ", version, flags, n, len(cols), ck) + bytes(24)
    assert len(head) == 64
    with open(path, "wb") as f:
        f.write(head + payload)


def _levels(d, g, roots):
    out = []
    lv = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for r in roots:
        g.run(int(r), lv)
        torch.cuda.synchronize()
        out.append(lv.cpu().numpy().copy())
    return np.stack(out)


@pytest.mark.parametrize("flags", [0, 0x2, 0x2 | 0x10, 0x20])
def test_round_trip(d, tmp_path, flags):
    spec = inputs.rmat(14)
    og = oracle.csr_from_rmat(spec)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 4, og.degrees() > 0)
    ref, _ = oracle.bfs_many(og, roots, want_parent=False)
    g = d.rmat_graph(spec, flags=flags)
    path = str(tmp_path / "g.dobfs")
    g.save(path)
    h = d.load_graph(path)
    a, b = g.info, h.info
    for f in ("n_vertices", "n_entries", "n_nonisolated", "max_degree", "offsets_int64", "reindexed"):
        assert getattr(a, f) == getattr(b, f), f
    for x, y in zip(g.export(), h.export()):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(h.degrees(), og.degrees())
    np.testing.assert_array_equal(_levels(d, h, roots), ref)
    # canonical parents are unique: equal to the oracle's
    lv = torch.empty(og.n, dtype=torch.int32, device="cuda")
    pa = torch.empty(og.n, dtype=torch.int32, device="cuda")
    _, ref_p = oracle.bfs_many(og, roots[:1])
    h.run(int(roots[0]), lv, pa, d.make_opts(flags=d.DOBFS_RUN_CANONICAL_PARENT))
    np.testing.assert_array_equal(pa.cpu().numpy(), ref_p[0])
    # batched runs on the loaded graph
    out = torch.empty((len(roots), og.n), dtype=torch.int32, device="cuda")
    d.dobfs_run_batch(h.handle, torch.from_numpy(np.ascontiguousarray(roots)).cuda(), out)
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    h.close()
    h = d.load_graph(path, validate=True)
    assert h.info.n_entries == og.nnz
    h.close()
    g.close()


def test_file_written_from_the_oracle_csr(d, tmp_path):
    """The documented layout, written here from the oracle's CSR (original
    IDs, int32 and int64 offsets), loads and gives the oracle's levels."""
    spec = inputs.rmat(11)
    og = oracle.csr_from_rmat(spec)
    roots = inputs.sample_roots(inputs.root_seed(spec.seed), og.n, 3, og.degrees() > 0)
    ref, _ = oracle.bfs_many(og, roots, want_parent=False)
    for off64 in (False, True):
        path = str(tmp_path / ("o%d.dobfs" % off64))
        _write_file(path, og.off, og.cols, off64=off64)
        g = d.load_graph(path, validate=True)
        assert g.info.offsets_int64 == int(off64) and g.info.reindexed == 0
        off, cols, n2o = g.export()
        np.testing.assert_array_equal(off, og.off)
        np.testing.assert_array_equal(cols, og.cols)
        np.testing.assert_array_equal(n2o, np.arange(og.n))
        np.testing.assert_array_equal(_levels(d, g, roots), ref)
        g.close()


def _small():
    # a path 0-1-2-3 plus a triangle 4-5-6 and an isolated vertex 7
    rows = {0: [1], 1: [0, 2], 2: [1, 3], 3: [2], 4: [5, 6], 5: [4, 6], 6: [4, 5], 7: []}
    off = np.zeros(9, dtype=np.int64)
    for v in range(8):
        off[v + 1] = off[v] + len(rows[v])
    cols = np.array([c for v in range(8) for c in rows[v]], dtype=np.int32)
    return off, cols


def _expect(d, path, status, validate=False):
    with pytest.raises(d.DobfsError) as e:
        d.load_graph(str(path), validate=validate)
    assert e.value.status == status, e.value


def test_damaged_files(d, tmp_path):
    off, cols = _small()
    good = tmp_path / "good.dobfs"
    _write_file(good, off, cols)
    g = d.load_graph(str(good), validate=True)
    lv = _levels(d, g, [0, 4, 7])
    np.testing.assert_array_equal(lv[0], [0, 1, 2, 3, -1, -1, -1, -1])
    np.testing.assert_array_equal(lv[1], [-1, -1, -1, -1, 0, 1, 1, -1])
    np.testing.assert_array_equal(lv[2], [-1] * 7 + [0])
    g.close()
    raw = good.read_bytes()
    cases = {
        "magic": b"NOTAGRPH" + raw[8:],
        "truncated": raw[:-8],
        "trailing": raw + bytes(8),
        "header_only": raw[:64],
        "short_header": raw[:20],
        "flipped": raw[:64 + 80] + bytes([raw[64 + 80] ^ 1]) + raw[64 + 81:],
    }
    for name, data in cases.items():
        p = tmp_path / (name + ".dobfs")
        p.write_bytes(data)
        _expect(d, p, d.DOBFS_ERR_IO)
    p = tmp_path / "version.dobfs"
    _write_file(p, off, cols, version=2)
    _expect(d, p, d.DOBFS_ERR_IO)
    p = tmp_path / "checksum.dobfs"
    _write_file(p, off, cols, checksum=12345)
    _expect(d, p, d.DOBFS_ERR_IO)
    _expect(d, tmp_path / "missing.dobfs", d.DOBFS_ERR_IO)
    with pytest.raises(d.DobfsError) as e:
        d.dobfs_graph_load(str(good), d.DOBFS_GRAPH_REINDEX)
    assert e.value.status == d.DOBFS_ERR_INVALID


def test_invariants_checked_on_load(d, tmp_path):
    off, cols = _small()

    def case(name, off_, cols_, n2o=None, status=None, validate=False):
        p = tmp_path / (name + ".dobfs")
        _write_file(p, off_, cols_, n2o=n2o)
        _expect(d, p, status or d.DOBFS_ERR_BAD_GRAPH, validate)

    c = cols.copy(); c[3] = 8
    case("col_range", off, c)
    c = cols.copy(); c[3] = -1
    case("col_negative", off, c)
    c = cols.copy(); c[1], c[2] = c[2], c[1]
    case("unsorted", off, c)
    c = cols.copy(); c[2] = 1                        # row 1 holds 0, 1: a self-loop
    case("self_loop", off, c)
    c = cols.copy(); c[6], c[7] = 5, 5               # row 4 holds 5 twice
    case("duplicate", off, c)
    o = off.copy(); o[3], o[4] = o[4], o[3]
    case("offsets", o, cols)
    o = off.copy(); o[-1] -= 1                       # offsets end before n_entries
    case("offsets_end", o, cols)
    # asymmetric (0 -> 1 kept, 1 -> 0 dropped): accepted unless validated
    o = off.copy(); o[2:] -= 1
    c = np.delete(cols, 1)
    p = tmp_path / "asym.dobfs"
    _write_file(p, o, c)
    d.load_graph(str(p)).close()
    _expect(d, p, d.DOBFS_ERR_BAD_GRAPH, validate=True)
    # renumbered graphs: the map must be a permutation and the degree classes
    # must not increase along the internal IDs
    deg = np.diff(off)
    order = np.lexsort((np.arange(8), -deg))         # by decreasing degree, ties by ID
    new_of = np.empty(8, dtype=np.int64); new_of[order] = np.arange(8)
    off_r = np.concatenate([[0], np.cumsum(deg[order])]).astype(np.int64)
    cols_r = np.concatenate([np.sort(new_of[cols[off[v]:off[v + 1]]]) for v in order]).astype(np.int32)
    p = tmp_path / "renumbered.dobfs"
    _write_file(p, off_r, cols_r, n2o=order)
    g = d.load_graph(str(p), validate=True)
    assert g.info.reindexed == 1
    np.testing.assert_array_equal(g.degrees(), deg)
    lv = _levels(d, g, [0, 5])
    np.testing.assert_array_equal(lv[0], [0, 1, 2, 3, -1, -1, -1, -1])
    np.testing.assert_array_equal(lv[1], [-1, -1, -1, -1, 1, 0, 1, -1])
    g.close()
    bad = order.copy(); bad[1] = bad[0]
    case("not_permutation", off_r, cols_r, n2o=bad)
    bad = order.copy(); bad[0] = 8
    case("map_range", off_r, cols_r, n2o=bad)
    # the original (not degree-sorted) CSR claimed as renumbered
    case("class_order", off, cols, n2o=np.arange(8))


def test_save_errors(d, tmp_path):
    off, cols = _small()
    p = tmp_path / "good.dobfs"
    _write_file(p, off, cols)
    g = d.load_graph(str(p))
    with pytest.raises(d.DobfsError) as e:
        g.save(str(tmp_path / "no_such_dir" / "x.dobfs"))
    assert e.value.status == d.DOBFS_ERR_IO
    with pytest.raises(d.DobfsError) as e:
        g.save(str(tmp_path))                        # a directory: not opened, not removed
    assert e.value.status == d.DOBFS_ERR_IO
    assert tmp_path.is_dir()
    g.close()
