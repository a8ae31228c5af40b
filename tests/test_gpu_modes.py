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
