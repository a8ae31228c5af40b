"""Query groups: the bound solves of up to eight same-type queries run as one
set of frontier rounds (one value lane per query), then each query's own
phases run from its lane.  Every output must equal the CPU oracle (and the
same query run alone), whatever the group size, the mix of windows and
sources, with and without pull rounds, and for the degenerate groups (one
source for every lane, isolated sources, one-snapshot windows)."""
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


def _specs(log, n, seed, types=(0, 1, 2, 3), hubs=None):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = int(rng.integers(1, log.S + 1))
        b = int(rng.integers(0, log.S - L + 1))
        src = int(hubs[k % len(hubs)]) if hubs is not None else int(rng.integers(0, log.V))
        out.append((types[k % len(types)], src, b, L))
    return out


def _hubs(log, n):
    deg = np.bincount(log.src[: log.n_base].astype(np.int64), minlength=log.V)
    return np.argsort(-deg, kind="stable")[:n]


def _run(svv, ctx, specs, gmax):
    ctx.set_tuning("batch_mode", 2)
    ctx.set_tuning("group_max", gmax)
    outs, st = ctx.query_batch(specs)
    assert st == [0] * len(specs)
    return outs


@pytest.mark.parametrize("gmax", [2, 4, 8])
def test_group_two_words_matches_oracle(svv, gmax):
    log = W.scaled_rmat(scale=12, edge_factor=8, n_snapshots=100, rate=0.003, seed=31, add_mode="skewed")
    specs = _specs(log, 26, 5 + gmax, hubs=_hubs(log, 9))
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        outs = _run(svv, ctx, specs, gmax)
        for (t, s, b, L), o in zip(specs, outs):
            np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, b, L))


@pytest.mark.parametrize("gmax", [2, 4, 8])
def test_mixed_type_groups_match_oracle(svv, gmax):
    """group_mix: queries of every type share a group's rounds, each lane in
    the min lattice with its own relaxation (SSWP on complemented widths);
    two mask words, hub and random sources, every window length."""
    log = W.scaled_rmat(scale=12, edge_factor=8, n_snapshots=100, rate=0.003, seed=37, add_mode="skewed")
    specs = _specs(log, 24, 70 + gmax, hubs=np.concatenate([_hubs(log, 6), np.arange(6) * 97]))
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        ctx.set_tuning("group_mix", 1)
        outs = _run(svv, ctx, specs, gmax)
        for (t, s, b, L), o in zip(specs, outs):
            np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, b, L))


@pytest.mark.parametrize("pull", [1, 0])
def test_mixed_pair_same_source(svv, pull):
    """An SSSP and an SSWP query from one hub over one window (two lanes, one
    of them complemented), with and without pull rounds, equal the queries
    alone and the oracle; weights up to 2^32 - 1 exercise the complement's
    edge cases (a weight of 0 complements to the identity)."""
    log = W.scaled_rmat(scale=14, edge_factor=16, n_snapshots=64, rate=0.001, seed=43)
    big = W.random_small_log(29, V=300, n_edges=3000, S=20, n_add=20, n_del=20, w_lo=0, w_hi=(1 << 32) - 1)
    for lg in (log, big):
        src = int(_hubs(lg, 1)[0])
        specs = [(0, src, 0, lg.S), (1, src, 0, lg.S), (3, src, 2, lg.S - 4), (2, src, 1, lg.S - 1)]
        with svv.Context(0) as ctx:
            ctx.set_tuning("pull", pull)
            ctx.load_log(lg)
            ctx.set_tuning("group_mix", 1)
            for n in (2, 4):
                outs = _run(svv, ctx, specs[:n], 8)
                for (t, s, b, L), o in zip(specs[:n], outs):
                    np.testing.assert_array_equal(svv.to_u32(o), oracle.query(lg, t, s, b, L))
                    assert torch.equal(o, ctx.query(t, s, b, L))


@pytest.mark.parametrize("pair", [(0, 1), (1, 1), (3, 3), (0, 3), (1, 2)])
def test_two_lane_groups_pull_every_round(svv, pair):
    """Two-lane groups (their own pull loop: four in-edges per lane, the run
    leader's target row loaded with the source rows), with both group solves
    pulling nearly every round; same-type pairs in their own lattice (SSWP's
    max lattice included) and mixed pairs in the min lattice."""
    log = W.scaled_rmat(scale=13, edge_factor=16, n_snapshots=70, rate=0.002, seed=47, add_mode="skewed")
    hubs = _hubs(log, 3)
    specs = [(pair[0], int(hubs[0]), 0, 70), (pair[1], int(hubs[1]), 5, 60)]
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        ctx.set_tuning("group_mix", 1)
        ctx.set_tuning("group_pull_pct", 1)
        ctx.set_tuning("group_pull_pct_union", 1)
        outs = _run(svv, ctx, specs, 2)
        for (t, s, b, L), o in zip(specs, outs):
            np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, b, L))


@pytest.mark.parametrize("pair", [(0, 0), (1, 1), (2, 2), (3, 3), (0, 1), (1, 3), (2, 0), (1, 2)])
def test_pair_tails_one_relaxation(svv, pair):
    """A two-query group whose windows have one length runs both relaxations
    as one launch over both queries' rows (a mixed pair in the min lattice,
    SSWP rows complemented); one and two mask words, results equal the oracle
    and the same pair with separate relaxations."""
    log = W.scaled_rmat(scale=13, edge_factor=8, n_snapshots=100, rate=0.003, seed=53, add_mode="skewed")
    hubs = _hubs(log, 4)
    # one context: the second pair's longer window grows the mask arrays
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        ctx.set_tuning("group_mix", 1)
        for L in (64, 100):
            specs = [(pair[0], int(hubs[0]), 0, L), (pair[1], int(hubs[1 + (L & 1)]), 100 - L, L)]
            ctx.set_tuning("pair_tails", 1)
            outs = _run(svv, ctx, specs, 2)
            for (t, s, b, L2), o in zip(specs, outs):
                np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, b, L2))
            # the bounds and row map of the batch's last query
            cap, cup, row = (torch.empty(log.V, dtype=torch.int32, device="cuda") for _ in range(3))
            svv.svv_get_bounds(ctx.h, cap, cup, row)
            t, s, b, L2 = specs[1]
            want_cap, want_cup = oracle.bounds(log, t, s, b, L2)
            np.testing.assert_array_equal(svv.to_u32(cap), want_cap)
            np.testing.assert_array_equal(svv.to_u32(cup), want_cup)
            assert np.array_equal(svv.to_u32(row) == 0xFFFFFFFF, want_cap == want_cup)
            ctx.set_tuning("pair_tails", 0)
            sep = _run(svv, ctx, specs, 2)
            for x, y in zip(outs, sep):
                assert torch.equal(x, y)


@pytest.mark.parametrize("pull", [1, 0])
def test_group_hubs_equal_alone(svv, pull):
    """Deep solves from hub sources (pull rounds when the frontier is large,
    or push only without the transposed graph)."""
    log = W.scaled_rmat(scale=15, edge_factor=16, n_snapshots=64, rate=0.0005, seed=41)
    specs = _specs(log, 24, 9, types=(0, 1, 2), hubs=_hubs(log, 12))
    with svv.Context(0) as ctx:
        ctx.set_tuning("pull", pull)
        ctx.load_log(log)
        outs = _run(svv, ctx, specs, 8)
        alone = ctx.empty_out(log.S)
        for (t, s, b, L), o in zip(specs, outs):
            ctx.query(t, s, b, L, out=alone[:L])
            assert torch.equal(o, alone[:L])
        for (t, s, b, L), o in list(zip(specs, outs))[:3]:
            np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, b, L))


def test_group_degenerate_lanes(svv):
    """One source and window in every lane; isolated sources; windows of one
    snapshot; the whole history; a group of the largest size next to a group
    of one."""
    log = W.small_rmat()
    deg = np.bincount(log.src.astype(np.int64), minlength=log.V)
    iso = int(np.flatnonzero(deg == 0)[0])
    hub = int(_hubs(log, 1)[0])
    specs = [(0, hub, 0, log.S)] * 8 + [(1, iso, 3, 1), (1, hub, 2, 1), (1, iso, 0, log.S)] + \
            [(2, hub, 0, 1), (2, hub, 7, 1)] + [(3, hub, 1, 5)]
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        outs = _run(svv, ctx, specs, 8)
        for (t, s, b, L), o in zip(specs, outs):
            np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, b, L))


def test_group_without_pruning(svv):
    """The no-pruning ablation (every vertex relaxed) through groups."""
    log = W.scaled_rmat(scale=11, edge_factor=8, n_snapshots=16, rate=0.01, seed=53)
    specs = _specs(log, 12, 3, hubs=_hubs(log, 4))
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        ctx.set_tuning("prune", 0)
        outs = _run(svv, ctx, specs, 4)
        for (t, s, b, L), o in zip(specs, outs):
            np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, b, L))


def test_group_host_outputs(svv):
    """Grouped instances with results in page-locked host memory."""
    log = W.scaled_rmat(scale=12, edge_factor=8, n_snapshots=40, rate=0.003, seed=61)
    specs = _specs(log, 10, 4, types=(0, 2), hubs=_hubs(log, 5))
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        ctx.set_tuning("group_max", 8)
        hosts = [torch.empty((L, log.V), dtype=torch.int32, pin_memory=True) for (_, _, _, L) in specs]
        st = svv.svv_query_batch(ctx.h, [(t, s, b, L, h) for (t, s, b, L), h in zip(specs, hosts)])
        assert st == [0] * len(specs)
        for (t, s, b, L), h in zip(specs, hosts):
            np.testing.assert_array_equal(h.numpy().view(np.uint32), oracle.query(log, t, s, b, L))


def test_group_bfs_levels_many_sources(svv):
    """BFS groups over many random sources on a larger graph, where a vertex
    can be in one lane's frontier while another lane's level of it is set in
    the same round; every level must still equal the query run alone."""
    log = W.scaled_rmat(scale=17, edge_factor=16, n_snapshots=64, rate=0.0005, seed=71)
    rng = np.random.default_rng(2)
    deg = np.bincount(log.src[: log.n_base].astype(np.int64), minlength=log.V)
    cand = np.flatnonzero(deg > 0)
    specs = []
    for k in range(24):
        L = int(rng.integers(8, 65))
        b = int(rng.integers(0, log.S - L + 1))
        specs.append((2, int(cand[rng.integers(0, cand.size)]), b, L))
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        outs = _run(svv, ctx, specs, 8)
        for (t, s, b, L), o in zip(specs, outs):
            assert torch.equal(o, ctx.query(t, s, b, L))
        for (t, s, b, L), o in list(zip(specs, outs))[:2]:
            np.testing.assert_array_equal(svv.to_u32(o)[[0, L - 1]],
                                          np.stack([oracle.query(log, t, s, b, 1)[0], oracle.query(log, t, s, b + L - 1, 1)[0]]))


def test_batch_graph_capture(svv):
    """Graph mode: an in-order batch's launches (group solves, member phases,
    status copies) are captured into one CUDA graph, updated in place for the
    next batch of the same shape, and replayed; results stay exact."""
    log = W.scaled_rmat(scale=13, edge_factor=8, n_snapshots=48, rate=0.003, seed=91)
    hubs = _hubs(log, 6)
    a = _specs(log, 14, 1, hubs=hubs)
    b = _specs(log, 14, 2, hubs=hubs)
    c = _specs(log, 9, 3)
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        ctx.set_tuning("graph", 1)
        for specs in (a, b, c, a):  # same shape twice, another shape, the first again
            outs = _run(svv, ctx, specs, 8)
            for (t, s, bb, L), o in zip(specs, outs):
                np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, s, bb, L))
