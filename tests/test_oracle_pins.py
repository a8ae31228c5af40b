"""Pins for the CPU oracle, against things other than itself.

* Floyd-Warshall brute force (min-plus, max-min, unit min-plus, min-max) on random
  multigraphs of <= 64 vertices with self-loops, sinks and unreachable parts.
* SciPy's Dijkstra / unweighted shortest paths on a 4,096-vertex RMAT snapshot.
* Widest path as a threshold-reachability closed form: the width of v is the
  largest t such that v is reachable from the source over edges of weight >= t;
  narrowest path likewise: the smallest t with v reachable over weights <= t.
* A pure-Python set replay of the edge log.
* Theorem 1 / Table 1 bounds and Theorem 2 (paper Section 3).
* Special cases (window of one snapshot, no deltas, isolated source, saturation).
* The hand-solved fixture under tests/golden/ (the paper's vertex-c numbers).
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse import csgraph

import oracle
import workloads as W

INF = 0xFFFFFFFF
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _csr(V, src, dst, w):
    order = np.argsort(src, kind="stable")
    rp = np.zeros(V + 1, np.uint64)
    np.add.at(rp, src.astype(np.int64) + 1, 1)
    rp = np.cumsum(rp).astype(np.uint64)
    return rp, dst[order].astype(np.uint32), w[order].astype(np.uint32)


def _fw(V, src, dst, w, kind):
    """Floyd-Warshall over the semiring of the query; returns V x V."""
    big = np.int64(1) << 40
    if kind == "ssnp":  # min-max semiring
        D = np.full((V, V), big, np.int64)
        for u, v, x in zip(src, dst, w.astype(np.int64)):
            D[u, v] = min(D[u, v], x)
        np.fill_diagonal(D, 0)
        for k in range(V):
            D = np.minimum(D, np.maximum(D[:, k:k + 1], D[k:k + 1, :]))
        return np.where(D >= big, INF, D).astype(np.uint64)
    if kind in ("sssp", "bfs"):
        D = np.full((V, V), big, np.int64)
        ww = np.ones_like(w, dtype=np.int64) if kind == "bfs" else w.astype(np.int64)
        for u, v, x in zip(src, dst, ww):
            D[u, v] = min(D[u, v], x)
        np.fill_diagonal(D, 0)
        for k in range(V):
            D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
        return np.where(D >= big, INF, D).astype(np.uint64)
    B = np.zeros((V, V), np.int64)
    for u, v, x in zip(src, dst, w.astype(np.int64)):
        B[u, v] = max(B[u, v], x)
    np.fill_diagonal(B, INF)
    for k in range(V):
        B = np.maximum(B, np.minimum(B[:, k:k + 1], B[k:k + 1, :]))
    return B.astype(np.uint64)


def _random_graph(rng, V, m, w_hi=50):
    src = rng.integers(0, V, m).astype(np.uint32)
    dst = rng.integers(0, V, m).astype(np.uint32)
    # leave a block of vertices with no in-edges from the rest (unreachable part)
    cut = V // 4
    bad = (dst < cut) & (src >= cut)
    dst[bad] = (dst[bad] + cut).astype(np.uint32)
    w = rng.integers(1, w_hi + 1, m).astype(np.uint32)
    # a few explicit self-loops and duplicate instances with other weights
    src[:3] = dst[:3]
    src[3:6], dst[3:6] = src[6:9], dst[6:9]
    return src, dst, w


@pytest.mark.parametrize("kind,qtype", [("sssp", oracle.SSSP), ("sswp", oracle.SSWP), ("bfs", oracle.BFS),
                                        ("ssnp", oracle.SSNP)])
@pytest.mark.parametrize("seed", range(6))
def test_floyd_warshall(kind, qtype, seed):
    rng = np.random.default_rng(100 + seed)
    V = int(rng.integers(5, 65))
    m = int(rng.integers(V, 4 * V))
    src, dst, w = _random_graph(rng, V, m)
    fw = _fw(V, src, dst, w, kind)
    rp, col, ww = _csr(V, src, dst, w)
    for s in sorted({0, V - 1, int(rng.integers(0, V))}):
        got = oracle.solve(qtype, V, rp, col, ww, s)
        np.testing.assert_array_equal(got.astype(np.uint64), fw[s])


@pytest.mark.parametrize("seed", range(6))
def test_widest_path_is_complemented_narrowest_path(seed):
    """The identity query groups of mixed types rely on: the widest-path width
    (max over paths of the min weight; 0 = unreachable, the source infinite)
    is the complement of the min over paths of the max COMPLEMENTED weight,
    i.e. SSWP(w) = ~SSNP(~w), with 0 and 2^32-1 among the weights."""
    rng = np.random.default_rng(300 + seed)
    V = int(rng.integers(5, 65))
    m = int(rng.integers(V, 4 * V))
    src, dst, _ = _random_graph(rng, V, m)
    w = rng.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32)
    w[: m // 8] = rng.choice(np.array([0, 1, 0xFFFFFFFE, 0xFFFFFFFF], np.uint32), m // 8)
    rp, col, ww = _csr(V, src, dst, w)
    for s in sorted({0, V - 1, int(rng.integers(0, V))}):
        wide = oracle.solve(oracle.SSWP, V, rp, col, ww, s)
        narrow_c = oracle.solve(oracle.SSNP, V, rp, col, ~ww, s)
        np.testing.assert_array_equal(wide, ~narrow_c)
        # and both against Floyd-Warshall over their own semirings
        np.testing.assert_array_equal(wide.astype(np.uint64), _fw(V, src, dst, w, "sswp")[s])


def _scipy_matrix(V, rp, col, w, unit=False):
    rows = np.repeat(np.arange(V), np.diff(rp.astype(np.int64)))
    ww = np.ones_like(w, dtype=np.float64) if unit else w.astype(np.float64)
    # multi-edges: keep the smallest weight (SciPy would add duplicates)
    key = rows.astype(np.int64) * V + col
    order = np.lexsort((ww, key))
    key, ww = key[order], ww[order]
    first = np.r_[True, key[1:] != key[:-1]]
    key, ww = key[first], ww[first]
    return sp.csr_matrix((ww, (key // V, key % V)), shape=(V, V))


@pytest.fixture(scope="module")
def small_log():
    return W.small_rmat()


def test_scipy_dijkstra_and_bfs(small_log):
    V = small_log.V
    rp, col, w = oracle.snapshot_csr(small_log, 3)
    M = _scipy_matrix(V, rp, col, w)
    for s in (0, 1, 77):
        ref = csgraph.dijkstra(M, directed=True, indices=s)
        ref = np.where(np.isinf(ref), INF, ref).astype(np.uint64)
        got = oracle.solve(oracle.SSSP, V, rp, col, w, s).astype(np.uint64)
        np.testing.assert_array_equal(got, ref)
        refb = csgraph.shortest_path(M, directed=True, unweighted=True, indices=s)
        refb = np.where(np.isinf(refb), INF, refb).astype(np.uint64)
        gotb = oracle.solve(oracle.BFS, V, rp, col, w, s).astype(np.uint64)
        np.testing.assert_array_equal(gotb, refb)


def test_widest_path_threshold_closed_form(small_log):
    V = small_log.V
    rp, col, w = oracle.snapshot_csr(small_log, 5)
    rows = np.repeat(np.arange(V), np.diff(rp.astype(np.int64)))
    for s in (0, 5):
        ref = np.zeros(V, np.uint64)
        for t in np.unique(w):  # ascending, so later (larger) t overwrite
            keep = w >= t
            A = sp.csr_matrix((np.ones(keep.sum()), (rows[keep], col[keep])), shape=(V, V))
            reach = csgraph.breadth_first_order(A, s, directed=True, return_predecessors=False)
            ref[reach] = t
        ref[s] = INF
        got = oracle.solve(oracle.SSWP, V, rp, col, w, s).astype(np.uint64)
        np.testing.assert_array_equal(got, ref)


def test_narrowest_path_threshold_closed_form(small_log):
    """SSNP value of v = the smallest t such that v is reachable from the
    source over edges of weight <= t (the source itself is 0)."""
    V = small_log.V
    rp, col, w = oracle.snapshot_csr(small_log, 4)
    rows = np.repeat(np.arange(V), np.diff(rp.astype(np.int64)))
    for s in (0, 9):
        ref = np.full(V, INF, np.uint64)
        for t in np.unique(w)[::-1]:  # descending, so later (smaller) t overwrite
            keep = w <= t
            A = sp.csr_matrix((np.ones(keep.sum()), (rows[keep], col[keep])), shape=(V, V))
            reach = csgraph.breadth_first_order(A, s, directed=True, return_predecessors=False)
            ref[reach] = t
        ref[s] = 0
        got = oracle.solve(oracle.SSNP, V, rp, col, w, s).astype(np.uint64)
        np.testing.assert_array_equal(got, ref)


def test_replay_matches_python_sets():
    for seed in range(3):
        log = W.random_small_log(seed, V=40, n_edges=120, S=6, n_add=9, n_del=7)
        alive = set()
        for snap in range(log.S):
            for k in log.del_ids[log.del_off[snap]:log.del_off[snap + 1]]:
                alive.discard(int(k))
            alive.update(range(int(log.add_off[snap]), int(log.add_off[snap + 1])))
            want = sorted((int(log.src[k]), int(log.dst[k]), int(log.w[k])) for k in alive)
            rp, col, w = oracle.snapshot_csr(log, snap)
            rows = np.repeat(np.arange(log.V), np.diff(rp.astype(np.int64)))
            got = sorted(zip(rows.tolist(), col.tolist(), w.tolist()))
            assert got == want
            # and the interval form of the same log
            live = [k for k in range(log.n_inst) if log.t_add[k] <= snap < log.t_del[k]]
            assert sorted(live) == sorted(alive)


def _python_alive(log):
    """Live instances of every snapshot, replaying the steps with Python sets
    (Section 2: a step's deletions, then its additions)."""
    alive, out = set(), []
    for snap in range(log.S):
        for k in log.del_ids[log.del_off[snap]:log.del_off[snap + 1]]:
            alive.discard(int(k))
        alive.update(range(int(log.add_off[snap]), int(log.add_off[snap + 1])))
        out.append(set(alive))
    return out


def _triples(log, keep):
    return sorted((int(log.src[k]), int(log.dst[k]), int(log.w[k])) for k in keep)


def _csr_triples(rp, col, w):
    rows = np.repeat(np.arange(rp.shape[0] - 1), np.diff(rp.astype(np.int64)))
    return sorted(zip(rows.tolist(), col.tolist(), w.tolist()))


def test_live_intervals_match_python_replay():
    for seed in range(4):
        log = W.random_small_log(seed, V=40, n_edges=120, S=7, n_add=9, n_del=7)
        t_add, t_del = oracle.live_intervals(log)
        for snap, alive in enumerate(_python_alive(log)):
            assert {k for k in range(log.n_inst) if t_add[k] <= snap < t_del[k]} == alive


def test_window_graphs_match_replay():
    """Every window's intersection / union graph from the intervals equals the
    intersection / union of the replayed snapshots, a one-snapshot window is
    the snapshot, and the bounds solved on them are oracle.bounds."""
    for seed in range(3):
        log = W.random_small_log(10 + seed, V=30, n_edges=90, S=6, n_add=8, n_del=8)
        iv = oracle.live_intervals(log)
        alive = _python_alive(log)
        rng = np.random.default_rng(seed)
        for b in range(log.S):
            for L in range(1, log.S - b + 1):
                cap_set = set.intersection(*alive[b:b + L])
                cup_set = set.union(*alive[b:b + L])
                rp_i, col_i, w_i = oracle.window_csr(log, iv, b, L, "cap")
                rp_u, col_u, w_u = oracle.window_csr(log, iv, b, L, "cup")
                assert _csr_triples(rp_i, col_i, w_i) == _triples(log, cap_set)
                assert _csr_triples(rp_u, col_u, w_u) == _triples(log, cup_set)
                if L == 1:
                    assert _csr_triples(*oracle.snapshot_csr(log, b)) == _triples(log, cap_set)
                qtype, src = int(rng.integers(0, 4)), int(rng.integers(0, log.V))
                cap, cup = oracle.bounds(log, qtype, src, b, L)
                np.testing.assert_array_equal(oracle.solve(qtype, log.V, rp_i, col_i, w_i, src), cap)
                np.testing.assert_array_equal(oracle.solve(qtype, log.V, rp_u, col_u, w_u, src), cup)


def _check_theorems(log, qtype, src, b, L):
    vals = oracle.query(log, qtype, src, b, L)
    cap, cup = oracle.bounds(log, qtype, src, b, L)
    if qtype == oracle.SSWP:  # Table 1: intersection <= G_i <= union
        assert (cap[None] <= vals).all() and (vals <= cup[None]).all()
    else:  # Theorem 1: union <= G_i <= intersection
        assert (cup[None] <= vals).all() and (vals <= cap[None]).all()
    stable = cap == cup
    # Theorem 2: a stable vertex has the same value in every snapshot
    assert (vals[:, stable] == cap[stable][None]).all()
    # safe but not complete: detected stable vertices are a subset of true UVVs
    uvv = (vals == vals[0:1]).all(axis=0)
    assert not (stable & ~uvv).any()
    return vals, cap, cup, stable, uvv


@pytest.mark.parametrize("qtype", [oracle.SSSP, oracle.SSWP, oracle.BFS, oracle.SSNP])
def test_theorems_small_rmat(small_log, qtype):
    for b, L in [(0, 8), (2, 5), (7, 1)]:
        vals, cap, cup, stable, uvv = _check_theorems(small_log, qtype, 0, b, L)
        if L == 1:  # G_cap = G_cup = G_b: everything is stable and equal
            assert stable.all()
            np.testing.assert_array_equal(vals[0], cap)


@pytest.mark.parametrize("seed", range(8))
def test_theorems_random(seed):
    rng = np.random.default_rng(seed)
    log = W.random_small_log(seed, V=int(rng.integers(8, 60)), n_edges=int(rng.integers(20, 200)),
                             S=int(rng.integers(1, 10)), n_add=int(rng.integers(0, 12)),
                             n_del=int(rng.integers(0, 12)))
    for qtype in (oracle.SSSP, oracle.SSWP, oracle.BFS, oracle.SSNP):
        L = int(rng.integers(1, log.S + 1))
        b = int(rng.integers(0, log.S - L + 1))
        _check_theorems(log, qtype, int(rng.integers(0, log.V)), b, L)


def test_no_deltas_everything_stable():
    log = W.random_small_log(5, V=50, n_edges=300, S=4, n_add=0, n_del=0)
    for qtype in (oracle.SSSP, oracle.SSWP, oracle.BFS, oracle.SSNP):
        vals, cap, cup, stable, _ = _check_theorems(log, qtype, 3, 0, 4)
        assert stable.all()
        assert (vals == cap[None]).all()


def test_isolated_source():
    log = W.random_small_log(9, V=30, n_edges=80, S=3, n_add=4, n_del=4)
    iso = 29
    keep = (log.src != iso)
    # re-route every out-edge of vertex 29 so it has none in any snapshot
    log.src = np.where(keep, log.src, 0).astype(np.uint32)
    for qtype, unreached in ((oracle.SSSP, INF), (oracle.SSWP, 0), (oracle.BFS, INF), (oracle.SSNP, INF)):
        vals = oracle.query(log, qtype, iso, 0, 3)
        other = np.arange(log.V) != iso
        assert (vals[:, other] == unreached).all()
        assert (vals[:, iso] == (INF if qtype == oracle.SSWP else 0)).all()


def test_bfs_equals_unit_weight_sssp(small_log):
    rp, col, w = oracle.snapshot_csr(small_log, 2)
    a = oracle.solve(oracle.BFS, small_log.V, rp, col, w, 0)
    b = oracle.solve(oracle.SSSP, small_log.V, rp, col, np.ones_like(w), 0)
    np.testing.assert_array_equal(a, b)


def test_sssp_saturates():
    # s -> a (0xFFFFFFF0), a -> b (0x100), b -> c (5): exact sums exceed 2^32-2
    rp = np.array([0, 1, 2, 3, 3], np.uint64)
    col = np.array([1, 2, 3], np.uint32)
    w = np.array([0xFFFFFFF0, 0x100, 5], np.uint32)
    got = oracle.solve(oracle.SSSP, 4, rp, col, w, 0)
    np.testing.assert_array_equal(got, [0, 0xFFFFFFF0, 0xFFFFFFFE, 0xFFFFFFFE])


class _Log:
    pass


def _golden_log():
    with open(os.path.join(GOLDEN, "vertex_c_example.json")) as f:
        g = json.load(f)
    lg = _Log()
    lg.V, lg.S = g["V"], g["S"]
    lg.src = np.array(g["src"], np.uint32)
    lg.dst = np.array(g["dst"], np.uint32)
    lg.w = np.array(g["w"], np.uint32)
    lg.add_off = np.array(g["add_off"], np.int64)
    lg.del_off = np.array(g["del_off"], np.int64)
    lg.del_ids = np.array(g["del_ids"], np.int64)
    return g, lg


@pytest.mark.parametrize("name,qtype", [("sssp", oracle.SSSP), ("sswp", oracle.SSWP), ("bfs", oracle.BFS),
                                        ("ssnp", oracle.SSNP)])
def test_golden_vertex_c(name, qtype):
    g, lg = _golden_log()
    exp = g["expected"][name]
    vals = oracle.query(lg, qtype, g["source"], 0, 2)
    np.testing.assert_array_equal(vals, np.array(exp["snapshots"], np.uint32))
    cap, cup = oracle.bounds(lg, qtype, g["source"], 0, 2)
    np.testing.assert_array_equal(cap, np.array(exp["cap"], np.uint32))
    np.testing.assert_array_equal(cup, np.array(exp["cup"], np.uint32))
    if name == "sssp":
        c = g["vertices"]["c"]
        assert (int(cup[c]), int(cap[c])) == (9, 11)
        assert vals[:, c].tolist() == [10, 10]


def test_bad_arguments_rejected():
    g, lg = _golden_log()
    with pytest.raises(ValueError):
        oracle.query(lg, oracle.SSSP, 99, 0, 1)
    with pytest.raises(ValueError):
        oracle.query(lg, oracle.SSSP, 0, 1, 2)
    with pytest.raises(ValueError):
        oracle.query(lg, 7, 0, 0, 1)
    with pytest.raises(ValueError):
        oracle.query(lg, 4, 0, 0, 1)
