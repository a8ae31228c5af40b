"""Compact output and the paper's ablation modes (Table 3): every mode must
give exactly the per-snapshot values of the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF


@pytest.fixture(scope="module")
def env():
    import __graft_entry__ as g
    g.build()
    from paper_2502_10579_gb300 import svv
    log = W.scaled_rmat(scale=13, edge_factor=8, n_snapshots=40, rate=0.003, seed=12)
    ctx = svv.Context(0)
    ctx.load_log(log)
    yield svv, log, ctx
    ctx.close()


@pytest.mark.parametrize("t", [0, 1, 2, 3])
def test_compact_output(env, t):
    svv, log, ctx = env
    for b, L in [(0, 40), (7, 13)]:
        V = log.V
        cap = torch.empty(V, dtype=torch.int32, device="cuda:0")
        row = torch.empty(V, dtype=torch.int32, device="cuda:0")
        rows = torch.empty(V * L, dtype=torch.int32, device="cuda:0")
        U = svv.svv_query_compact(ctx.h, t, 0, b, L, cap, row, rows)
        capn, rown = svv.to_u32(cap), svv.to_u32(row)
        rowsn = svv.to_u32(rows)[: U * L].reshape(U, L)
        stable = rown == INF
        assert int((~stable).sum()) == U
        full = np.where(stable[None, :], capn[None, :], rowsn[np.where(stable, 0, rown)].T)
        np.testing.assert_array_equal(full, oracle.query(log, t, 0, b, L))
        # too small a rows buffer is refused
        if U:
            small = torch.empty(max(U * L - 1, 1), dtype=torch.int32, device="cuda:0")
            with pytest.raises(svv.SvvError) as e:
                svv.svv_query_compact(ctx.h, t, 0, b, L, cap, row, small)
            assert e.value.status == 2


@pytest.mark.parametrize("knobs", [{"slab_max": 1}, {"prune": 0}, {"prune": 0, "slab_max": 1}, {"slab_max": 5}])
def test_ablation_modes_exact(env, knobs):
    svv, log, ctx = env
    try:
        for k, v in knobs.items():
            ctx.set_tuning(k, v)
        for t in (0, 1, 2):
            np.testing.assert_array_equal(svv.to_u32(ctx.query(t, 3, 2, 30)), oracle.query(log, t, 3, 2, 30))
        if knobs.get("prune") == 0:
            assert ctx.stats()["unstable"] == log.V  # no pruning: every vertex relaxed
    finally:
        ctx.set_tuning("slab_max", 128)
        ctx.set_tuning("prune", 1)


@pytest.fixture(scope="module")
def env2():
    """Two mask words, a skewed degree mix and a hub source, so that frontiers
    grow past the pull threshold."""
    import __graft_entry__ as g
    g.build()
    from paper_2502_10579_gb300 import svv
    log = W.scaled_rmat(scale=14, edge_factor=16, n_snapshots=90, rate=0.002, seed=33, add_mode="skewed")
    return svv, log, W.max_out_degree_vertex(log)


_want = {}


def _oracle(log, t, src, b, L):
    key = (id(log), t, src, b, L)
    if key not in _want:
        _want[key] = oracle.query(log, t, src, b, L)
    return _want[key]


@pytest.mark.parametrize("knobs", [
    {"pull_pct": 0},                                   # push rounds only
    {"pull_pct": 1},                                   # pull almost every round
    {"skip_same": 0},
    {"delta_sssp": 40, "delta_sswp": 40},              # near-far deferral
    {"relax_lanes": 8}, {"relax_lanes": 16},
    {"graph": 1},
])
def test_solver_knobs_exact(env2, knobs):
    """Every launch knob changes only the work, never the values."""
    svv, log, src = env2
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        for k, v in knobs.items():
            ctx.set_tuning(k, v)
        for t in (0, 1, 2, 3):
            for b, L in [(0, 90), (10, 70)]:
                np.testing.assert_array_equal(svv.to_u32(ctx.query(t, src, b, L)), _oracle(log, t, src, b, L))


@pytest.mark.parametrize("knobs", [
    {"solve_chunk": 16, "relax_chunk": 8, "qrs_chunk": 64},
    {"solve_chunk": 256, "relax_chunk": 128, "qrs_chunk": 1024},
    {"pull": 0},                                       # no transposed graph
])
def test_load_time_knobs_exact(env2, knobs):
    """Knobs fixed when the graph is loaded (chunk sizes, the transposed
    graph) change only the work."""
    svv, log, src = env2
    with svv.Context(0) as ctx:
        for k, v in knobs.items():
            ctx.set_tuning(k, v)
        ctx.load_log(log)
        for t in (0, 1, 2, 3):
            np.testing.assert_array_equal(svv.to_u32(ctx.query(t, src, 5, 80)), _oracle(log, t, src, 5, 80))


@pytest.mark.parametrize("t", [0, 1, 2, 3])
def test_isolated_source_fast_path(env, t):
    """A source with no out-edge in any snapshot is answered by one fill: the
    result, the bounds (svv_get_bounds) and the compact form must equal the
    oracle and the full pipeline (isolated_fast = 0)."""
    svv, log, ctx = env
    deg = np.bincount(log.src.astype(np.int64), minlength=log.V)
    iso = int(np.flatnonzero(deg == 0)[0])
    for b, L in [(0, 40), (11, 1), (5, 31)]:
        want = oracle.query(log, t, iso, b, L)
        fast = svv.to_u32(ctx.query(t, iso, b, L))
        np.testing.assert_array_equal(fast, want)
        cap, cup, row = ctx.bounds()
        ocap, ocup = oracle.bounds(log, t, iso, b, L)
        np.testing.assert_array_equal(cap, ocap)
        np.testing.assert_array_equal(cup, ocup)
        assert (row == INF).all() and ctx.stats()["unstable"] == 0
        ctx.set_tuning("isolated_fast", 0)
        try:
            np.testing.assert_array_equal(svv.to_u32(ctx.query(t, iso, b, L)), want)
        finally:
            ctx.set_tuning("isolated_fast", 1)
        capt = torch.empty(log.V, dtype=torch.int32, device="cuda:0")
        rowt = torch.empty(log.V, dtype=torch.int32, device="cuda:0")
        rows = torch.empty(4, dtype=torch.int32, device="cuda:0")
        assert svv.svv_query_compact(ctx.h, t, iso, b, L, capt, rowt, rows) == 0
        np.testing.assert_array_equal(svv.to_u32(capt), ocap)
