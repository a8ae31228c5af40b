"""The seeded input generators: deterministic, consistent edge logs with the
sizes, weight ranges, churn and query mixes the workloads are defined by."""
import numpy as np
import pytest

import workloads as W


def _check_log(log, n_add=None, n_del=None, w_lo=None, w_hi=None):
    S, n = log.S, log.n_inst
    assert log.add_off.shape == (S + 1,) and log.del_off.shape == (S + 1,)
    assert log.add_off[0] == 0 and log.add_off[-1] == n and log.del_off[0] == 0 and log.del_off[1] == 0
    assert np.all(np.diff(log.add_off) >= 0) and np.all(np.diff(log.del_off) >= 0)
    assert log.src.max(initial=0) < log.V and log.dst.max(initial=0) < log.V
    # t_add is the step that added the instance
    steps = np.repeat(np.arange(S), np.diff(log.add_off))
    np.testing.assert_array_equal(log.t_add, steps)
    # every deletion removes a live instance once, and t_del records the step
    assert np.unique(log.del_ids).shape == log.del_ids.shape
    t_del = np.full(n, S, np.int64)
    for s in range(1, S):
        ids = log.del_ids[log.del_off[s]:log.del_off[s + 1]]
        assert np.all(log.t_add[ids] < s)  # added before, so live until now
        t_del[ids] = s
    np.testing.assert_array_equal(log.t_del, t_del)
    assert np.all(log.t_add < log.t_del)
    if n_add is not None:
        assert np.all(np.diff(log.add_off)[1:] == n_add)
    if n_del is not None:
        assert np.all(np.diff(log.del_off)[1:] == n_del)
    if w_lo is not None:
        assert log.w.min() >= w_lo and log.w.max() <= w_hi


def test_small_rmat_recipe_and_determinism():
    a, b = W.small_rmat(), W.small_rmat()
    for f in ("src", "dst", "w", "add_off", "del_off", "del_ids", "t_add", "t_del"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert (a.V, a.S, a.n_base) == (4096, 8, 32768)
    _check_log(a, n_add=328, n_del=328, w_lo=1, w_hi=255)
    c = W.small_rmat(seed=7)
    assert not np.array_equal(a.src, c.src)


def test_rmat20_recipe():
    log = W.rmat20()
    assert (log.V, log.S, log.n_base) == (1 << 20, 64, 1 << 24)
    _check_log(log, n_add=10000, n_del=10000, w_lo=1, w_hi=999)
    # RMAT skew: a few vertices hold a large share of the out-edges
    deg = np.bincount(log.src[: log.n_base].astype(np.int64), minlength=log.V)
    assert deg.max() > 50 * deg.mean()
    assert deg[W.max_out_degree_vertex(log)] == deg.max()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_small_logs(seed):
    log = W.random_small_log(seed, V=50, n_edges=200, S=9, n_add=5, n_del=7, w_lo=3, w_hi=9)
    _check_log(log, n_add=5, n_del=7, w_lo=3, w_hi=9)


def test_max_out_degree_vertex_ties_take_smallest_id():
    log = W.random_small_log(4, V=6, n_edges=0, S=2, n_add=0, n_del=0)
    log.src = np.array([3, 3, 1, 1, 5], np.uint32)
    log.dst = np.zeros(5, np.uint32)
    log.add_off = np.array([0, 5, 5], np.int64)
    assert W.max_out_degree_vertex(log) == 1


def test_query_mixes():
    log = W.small_rmat()
    qs = W.batch_queries(log, n=90, seed=3, l_lo=2, l_hi=8)
    types = [q.type for q in qs]
    assert sorted(set(types)) == [W.SSSP, W.SSWP, W.BFS] and types.count(W.SSSP) == 30
    assert all(2 <= q.win_len <= 8 and q.win_begin + q.win_len <= log.S and q.source < log.V for q in qs)
    reqs = W.serve_requests(log, rate=200.0, duration_s=0.5, seed=5, l_lo=2, l_hi=8)
    arr = [a for a, _ in reqs]
    assert arr == sorted(arr) and 0 < arr[-1] < 0.5 and 50 < len(reqs) < 200
    assert all(q.win_begin + q.win_len <= log.S for _, q in reqs)
    q24 = W.rmat24_queries(log, n_sources=4, seed=4, windows=(2, 4, 8))
    assert len(q24) == 24 and {q.type for q in q24} == {W.SSSP, W.BFS}
    deg = np.bincount(log.src[: log.n_base].astype(np.int64), minlength=log.V)
    assert all(deg[q.source] > 0 and q.win_begin == 0 for q in q24)
