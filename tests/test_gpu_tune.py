"""Autotuner: picks per-type, per-window-length knobs by timing a probe query
(pull threshold, near-far width, work-unit size, CTAs per SM, relaxation lanes,
chunk skipping, slab width); results stay exact."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotune_keeps_results_exact():
    import __graft_entry__ as g
    g.build()
    from paper_2502_10579_gb300 import svv
    log = W.scaled_rmat(scale=14, edge_factor=8, n_snapshots=32, rate=0.002, seed=21)
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        for t in (0, 2):
            r = svv.svv_autotune(ctx.h, t, 0, 0, log.S, reps=2)
            assert r["candidates"] >= 2
            assert r["solve_chunk"] in (32, 64) and r["relax_lanes"] in (16, 32)
            assert r["pull_pct"] in (0, 5, 10, 15, 25, 40) and r["slab_max"] in (128, 64, 32)
            assert r["delta"] in ((0, 250, 1000, 4000) if t == 0 else (0,))
            assert 0 < r["best_ms"] <= r["default_ms"]
            for b, L in [(0, log.S), (5, 9)]:
                np.testing.assert_array_equal(svv.to_u32(ctx.query(t, 3, b, L)), oracle.query(log, t, 3, b, L))


def test_graph_mode_replays_exactly():
    import __graft_entry__ as g
    g.build()
    from paper_2502_10579_gb300 import svv
    log = W.scaled_rmat(scale=12, edge_factor=8, n_snapshots=140, rate=0.003, seed=8)
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        ctx.set_tuning("graph", 1)
        # same shape twice (graph updated in place), then other shapes
        for t, s, b, L in [(0, 1, 0, 64), (0, 9, 3, 64), (1, 2, 10, 40), (3, 5, 0, 140), (2, 7, 1, 139), (0, 1, 0, 64)]:
            np.testing.assert_array_equal(svv.to_u32(ctx.query(t, s, b, L)), oracle.query(log, t, s, b, L))
