"""Long solves: a path keeps the frontier at one vertex for thousands of
rounds, each ended by a team barrier; with a short barrier limit (4 ms) every
barrier must still complete, and the values must equal the oracle's."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _path_log(V=3000, S=4):
    """A path 0 -> 1 -> ... -> V-1 (weights 1..9) in every snapshot, plus a
    few changes: step 1 deletes edge 1000 -> 1001 and adds 999 -> 1001, step 2
    adds a shortcut 0 -> 2500."""
    rng = np.random.default_rng(5)
    src = list(range(V - 1))
    dst = list(range(1, V))
    w = [int(x) for x in rng.integers(1, 10, size=V - 1)]
    n_base = V - 1
    src += [999, 0]
    dst += [1001, 2500]
    w += [5, 7]
    t_add = [0] * n_base + [1, 2]
    t_del = [S] * (n_base + 2)
    t_del[1000] = 1
    add_off = [0, n_base, n_base + 1, n_base + 2] + [n_base + 2] * (S - 3)
    del_off = [0, 0, 1, 1] + [1] * (S - 3)
    return W.EdgeLog(V=V, S=S, src=np.array(src, np.uint32), dst=np.array(dst, np.uint32),
                     w=np.array(w, np.uint32), add_off=np.array(add_off, np.int64),
                     del_off=np.array(del_off, np.int64), del_ids=np.array([1000], np.int64),
                     t_add=np.array(t_add, np.uint32), t_del=np.array(t_del, np.uint32))


def test_path_thousands_of_rounds():
    import __graft_entry__ as g
    g.build()
    from paper_2502_10579_gb300 import svv
    log = _path_log()
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        ctx.set_tuning("spin_limit_ms", 4)
        for t in (0, 1, 2, 3):
            for b, L in [(0, 4), (1, 2)]:
                np.testing.assert_array_equal(svv.to_u32(ctx.query(t, 0, b, L)), oracle.query(log, t, 0, b, L))
        assert ctx.stats()["iters_cap"] > 1000  # the path's rounds did run
        ctx.set_tuning("spin_limit_ms", 1000)
