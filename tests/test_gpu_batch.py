"""Batched queries in one persistent launch (svv_query_batch): every instance
must equal the CPU oracle, and equal the same query run alone."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def svv():
    import __graft_entry__ as g
    g.build()
    from paper_2502_10579_gb300 import svv as mod
    assert torch.cuda.is_available()
    return mod


def _mixed(log, n, seed, l_lo=1, l_hi=None):
    rng = np.random.default_rng(seed)
    l_hi = l_hi or log.S
    out = []
    for k in range(n):
        L = int(rng.integers(l_lo, l_hi + 1))
        b = int(rng.integers(0, log.S - L + 1))
        out.append((k % 4, int(rng.integers(0, log.V)), b, L))
    return out


def test_batch_small_matches_oracle(svv):
    log = W.small_rmat()
    specs = _mixed(log, 30, 1) + [(0, 0, 0, 8), (1, 0, 0, 8), (2, 0, 0, 8)]
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        outs, st = ctx.query_batch(specs)
        assert st == [0] * len(specs)
        for (t, s, b, L), o in zip(specs, outs):
            np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, b, L))
        assert ctx.stats()["batch_teams"] >= 1


@pytest.mark.parametrize("teams", [1, 3, 8])
def test_batch_teams_and_two_words(svv, teams):
    log = W.scaled_rmat(scale=13, edge_factor=8, n_snapshots=100, rate=0.003, seed=91, add_mode="skewed")
    specs = _mixed(log, 20, 7 + teams)
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        ctx.set_tuning("batch_teams", teams)
        outs, st = ctx.query_batch(specs)
        assert st == [0] * len(specs)
        for (t, s, b, L), o in zip(specs, outs):
            alone = svv.to_u32(ctx.query(t, s, b, L))
            np.testing.assert_array_equal(svv.to_u32(o), alone)
        # pin two instances to the oracle as well
        for (t, s, b, L), o in list(zip(specs, outs))[:2]:
            np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, b, L))


def test_batch_in_order_mode(svv):
    """batch_mode 2 runs the instances one after another with svv_query's
    kernels; results and per-spec statuses are the same as in one launch."""
    log = W.scaled_rmat(scale=12, edge_factor=8, n_snapshots=100, rate=0.003, seed=17, add_mode="skewed")
    specs = _mixed(log, 12, 21) + [(3, 1, 0, 100)]
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        ctx.set_tuning("batch_mode", 2)
        outs, st = ctx.query_batch(specs)
        assert st == [0] * len(specs)
        assert ctx.stats()["batch_teams"] == 0
        for (t, s, b, L), o in zip(specs, outs):
            np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, b, L))
        good = ctx.empty_out(4)
        st = svv.svv_query_batch(ctx.h, [(0, log.V, 0, 4, good), (1, 0, 0, 4, good)])
        assert st == [1, 0]
        np.testing.assert_array_equal(svv.to_u32(good), oracle.query(log, 1, 0, 0, 4))


def test_batch_invalid_spec_is_skipped(svv):
    log = W.small_rmat()
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        good = ctx.empty_out(4)
        bad = ctx.empty_out(4)
        st = svv.svv_query_batch(ctx.h, [(0, 0, 0, 4, good), (0, log.V + 5, 0, 4, bad), (7, 0, 0, 4, bad)])
        assert st == [0, 1, 1]
        np.testing.assert_array_equal(svv.to_u32(good), oracle.query(log, 0, 0, 0, 4))


def test_batch_under_a_tight_budget(svv):
    log = W.scaled_rmat(scale=12, edge_factor=8, n_snapshots=16, rate=0.01, seed=3)
    specs = _mixed(log, 12, 5)
    with svv.Context(0) as roomy:
        roomy.load_log(log)
        want = [svv.to_u32(roomy.query(t, s, b, L)) for t, s, b, L in specs]
        graph_and_query = roomy.device_bytes()
    # room for the graph, the single-query scratch and about one batch team
    with svv.Context(0, hbm_budget_bytes=int(graph_and_query * 1.9)) as ctx:
        ctx.load_log(log)
        ctx.set_tuning("batch_teams", 8)
        outs, st = ctx.query_batch(specs)
        assert st == [0] * len(specs)
        assert 1 <= ctx.stats()["batch_teams"] < 8
        for w, o in zip(want, outs):
            np.testing.assert_array_equal(svv.to_u32(o), w)


def test_batch_config3_shape(svv):
    """The mixed batch workload, scaled down: RMAT scale 16, 64 snapshots,
    0.05% churn per step, 64 queries of 1/3 SSSP, SSWP, BFS with window
    lengths uniform in [8, 64] at uniform offsets."""
    log = W.scaled_rmat(scale=16, edge_factor=16, n_snapshots=64, rate=0.0005, seed=1003)
    qs = W.batch_queries(log, n=64, seed=3)
    specs = [(q.type, q.source, q.win_begin, q.win_len) for q in qs]
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        outs, st = ctx.query_batch(specs)
        assert st == [0] * len(specs)
        for (t, s, b, L), o in zip(specs, outs):
            np.testing.assert_array_equal(svv.to_u32(o), svv.to_u32(ctx.query(t, s, b, L)))
        for (t, s, b, L), o in list(zip(specs, outs))[:3]:
            np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, b, L))


def test_batch_host_outputs(svv):
    """Host outputs (page-locked and pageable) in a batch: computed into
    staging slots and copied back while the next instance computes."""
    log = W.scaled_rmat(scale=12, edge_factor=8, n_snapshots=70, rate=0.004, seed=23, add_mode="skewed")
    specs = _mixed(log, 7, 31)
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        outs = []
        for k, (t, s, b, L) in enumerate(specs):
            if k % 3 == 0:
                outs.append(torch.empty((L, log.V), dtype=torch.int32, pin_memory=True))
            elif k % 3 == 1:
                outs.append(np.empty((L, log.V), np.uint32))
            else:
                outs.append(ctx.empty_out(L))
        st = svv.svv_query_batch(ctx.h, [sp + (o,) for sp, o in zip(specs, outs)])
        assert st == [0] * len(specs)
        for (t, s, b, L), o in zip(specs, outs):
            got = o if isinstance(o, np.ndarray) else svv.to_u32(o) if o.is_cuda else o.numpy().view(np.uint32)
            np.testing.assert_array_equal(got, oracle.query(log, t, s, b, L))
