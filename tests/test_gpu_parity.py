"""GPU parity: the library's CUDA path against the CPU oracle, bit for bit.

Every check calls through the C ABI (ctypes binding).  Values are exact uint32
lattice values, so the only correct agreement is equality.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF
TYPES = (0, 1, 2, 3)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def svv():
    import __graft_entry__ as g
    g.build()
    from paper_2502_10579_gb300 import svv as mod
    assert torch.cuda.is_available()
    return mod


@pytest.fixture(scope="module")
def small(svv):
    log = W.small_rmat()
    ctx = svv.Context(0)
    ctx.load_log(log)
    yield log, ctx
    ctx.close()


def _iu(svv, ctx, t, s, b, L):
    return svv.to_u32(ctx.query(t, s, b, L))


def _plain(svv, ctx, t, s, b, L):
    return svv.to_u32(ctx.query(t, s, b, L, plain=True))


@pytest.mark.parametrize("t", TYPES)
def test_small_rmat_full(svv, small, t):
    log, ctx = small
    for src in (0, 1, 123):
        for b, L in [(0, 8), (2, 5), (7, 1), (0, 1), (3, 4)]:
            want = oracle.query(log, t, src, b, L)
            np.testing.assert_array_equal(_iu(svv, ctx, t, src, b, L), want)
            np.testing.assert_array_equal(_plain(svv, ctx, t, src, b, L), want)


@pytest.mark.parametrize("t", TYPES)
def test_small_rmat_steps(svv, small, t):
    """Intersection/union bounds (Section 3 Step 1) and the stable set (Step 2)."""
    log, ctx = small
    for b, L in [(0, 8), (1, 6)]:
        _iu(svv, ctx, t, 0, b, L)
        cap, cup, row = ctx.bounds()
        ocap, ocup = oracle.bounds(log, t, 0, b, L)
        np.testing.assert_array_equal(cap, ocap)
        np.testing.assert_array_equal(cup, ocup)
        stable = ocap == ocup
        assert ((row == INF) == stable).all()
        rows = row[~stable]
        assert sorted(rows.tolist()) == list(range(int((~stable).sum())))
        assert (np.diff(rows.astype(np.int64)) > 0).all()  # rows in vertex order
        st = ctx.stats()
        assert st["unstable"] == int((~stable).sum())


def test_golden_vertex_c(svv):
    with open(os.path.join(GOLDEN, "vertex_c_example.json")) as f:
        g = json.load(f)
    src = np.array(g["src"], np.uint32)
    t_add = np.zeros(len(src), np.uint32)
    t_del = np.full(len(src), g["S"], np.uint32)
    for s in range(1, g["S"]):
        t_add[g["add_off"][s]:g["add_off"][s + 1]] = s
        for k in g["del_ids"][g["del_off"][s]:g["del_off"][s + 1]]:
            t_del[k] = s
    rp, col, w, mask = svv.svv_build_versioned_csr(g["V"], g["S"], src, np.array(g["dst"], np.uint32),
                                                   np.array(g["w"], np.uint32), t_add, t_del)
    with svv.Context(0) as ctx:
        ctx.load_csr(g["V"], g["S"], rp, col, w, mask)
        for name, t in (("sssp", 0), ("sswp", 1), ("bfs", 2), ("ssnp", 3)):
            exp = g["expected"][name]
            got = _iu(svv, ctx, t, g["source"], 0, 2)
            np.testing.assert_array_equal(got, np.array(exp["snapshots"], np.uint32))
            cap, cup, row = ctx.bounds()
            np.testing.assert_array_equal(cap, np.array(exp["cap"], np.uint32))
            np.testing.assert_array_equal(cup, np.array(exp["cup"], np.uint32))


@pytest.mark.parametrize("seed", range(10))
def test_random_logs(svv, seed):
    rng = np.random.default_rng(500 + seed)
    S = int(rng.choice([1, 2, 5, 64, 65, 100, 130, 200]))
    log = W.random_small_log(seed, V=int(rng.integers(2, 300)), n_edges=int(rng.integers(0, 1500)),
                             S=S, n_add=int(rng.integers(0, 20)), n_del=int(rng.integers(0, 20)),
                             w_hi=int(rng.choice([1, 5, 1000])))
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        for t in TYPES:
            for _ in range(3):
                L = int(rng.integers(1, S + 1))
                b = int(rng.integers(0, S - L + 1))
                src = int(rng.integers(0, log.V))
                want = oracle.query(log, t, src, b, L)
                np.testing.assert_array_equal(_iu(svv, ctx, t, src, b, L), want)
                if L <= 70:
                    np.testing.assert_array_equal(_plain(svv, ctx, t, src, b, L), want)


def test_saturating_weights(svv):
    """Weights near 2^32: SSSP sums saturate at 0xFFFFFFFE (never reaching the
    unreachable code), SSWP/SSNP bottlenecks take the huge weights as they are."""
    log = W.random_small_log(17, V=150, n_edges=900, S=70, n_add=12, n_del=12, w_lo=1 << 30,
                             w_hi=(1 << 32) - 1)
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        for t in TYPES:
            for src, b, L in [(0, 0, 70), (5, 3, 40), (9, 60, 10)]:
                want = oracle.query(log, t, src, b, L)
                if t == 0:
                    assert (want == 0xFFFFFFFE).any()  # the case is exercised
                np.testing.assert_array_equal(_iu(svv, ctx, t, src, b, L), want)
                np.testing.assert_array_equal(_plain(svv, ctx, t, src, b, L), want)


@pytest.fixture(scope="module")
def medium(svv):
    # scale-14 RMAT, 100 snapshots (two mask words), degree-skewed additions
    log = W.scaled_rmat(scale=14, edge_factor=8, n_snapshots=100, rate=0.002, seed=77, add_mode="skewed")
    ctx = svv.Context(0)
    ctx.load_log(log)
    yield log, ctx
    ctx.close()


@pytest.mark.parametrize("t", TYPES)
def test_medium_two_words(svv, medium, t):
    log, ctx = medium
    src = W.max_out_degree_vertex(log)
    for b, L in [(0, 100), (10, 50), (37, 27), (60, 40), (99, 1)]:
        want = oracle.query(log, t, src, b, L)
        np.testing.assert_array_equal(_iu(svv, ctx, t, src, b, L), want)
    np.testing.assert_array_equal(_plain(svv, ctx, t, src, 40, 24), oracle.query(log, t, src, 40, 24))


def test_every_window_length(svv, medium):
    """Every window length 1..100 once (the output tile, the relaxation rows
    and the mask words change size at different lengths; 95 and 96 snapshots
    once put the tile just past the default shared-memory limit)."""
    log, ctx = medium
    src = W.max_out_degree_vertex(log)
    rng = np.random.default_rng(5)
    out = ctx.empty_out(log.S)
    for L in range(1, log.S + 1):
        b = int(rng.integers(0, log.S - L + 1))
        t = TYPES[L % len(TYPES)]
        ctx.query(t, src, b, L, out=out[:L])
        got = svv.to_u32(out[:L])
        # the first and last snapshot against the oracle (every snapshot for
        # the lengths where a size changes)
        if L in (1, 63, 64, 65, 94, 95, 96, 97, 100):
            np.testing.assert_array_equal(got, oracle.query(log, t, src, b, L))
        else:
            for i in (0, L - 1):
                np.testing.assert_array_equal(got[i], oracle.query(log, t, src, b + i, 1)[0])


def test_long_window_slabs(svv):
    # windows longer than one 128-snapshot slab
    log = W.scaled_rmat(scale=10, edge_factor=8, n_snapshots=300, rate=0.004, seed=5)
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        for t in TYPES:
            for b, L in [(0, 300), (17, 200), (100, 129)]:
                np.testing.assert_array_equal(_iu(svv, ctx, t, 0, b, L), oracle.query(log, t, 0, b, L))


def test_degenerate_graphs(svv):
    with svv.Context(0) as ctx:
        # one vertex, no edges
        ctx.load_csr(1, 3, np.zeros(2, np.uint64), np.zeros(0, np.uint32), np.zeros(0, np.uint32),
                     np.zeros(0, np.uint64))
        for t, v in ((0, 0), (1, INF), (2, 0), (3, 0)):
            assert _iu(svv, ctx, t, 0, 0, 3).tolist() == [[v]] * 3
        # edges present in no snapshot are dropped; self-loops and multi-edges kept
        rp = np.array([0, 3, 4, 4], np.uint64)
        col = np.array([1, 0, 1, 2], np.uint32)
        w = np.array([5, 1, 3, 2], np.uint32)
        mask = np.array([0b11, 0b11, 0b10, 0b00], np.uint64)
        ctx.load_csr(3, 2, rp, col, w, mask)
        np.testing.assert_array_equal(_iu(svv, ctx, 0, 0, 0, 2), [[0, 5, INF], [0, 3, INF]])
        np.testing.assert_array_equal(_iu(svv, ctx, 1, 0, 0, 2), [[INF, 5, 0], [INF, 5, 0]])


def test_isolated_source_and_no_deltas(svv):
    log = W.random_small_log(1, V=200, n_edges=300, S=6, n_add=0, n_del=0)
    isolated = np.setdiff1d(np.arange(log.V), log.src)
    assert isolated.size > 0
    iso = int(isolated[0])
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        for t in TYPES:
            np.testing.assert_array_equal(_iu(svv, ctx, t, iso, 0, 6), oracle.query(log, t, iso, 0, 6))
            _iu(svv, ctx, t, 0, 0, 6)
            assert ctx.stats()["unstable"] == 0  # no deltas: every vertex is stable


def test_inputs_on_device_and_host_output(svv, small):
    log, _ = small
    rp, col, w, mask = svv.svv_build_versioned_csr(log.V, log.S, log.src, log.dst, log.w, log.t_add, log.t_del)
    d = [torch.from_numpy(x.view(np.int64) if x.dtype == np.uint64 else x.view(np.int32)).cuda()
         for x in (rp, col, w, mask)]
    with svv.Context(0) as ctx:
        ctx.load_csr(log.V, log.S, *d, inputs_on_device=True)
        host = np.empty((log.S, log.V), np.uint32)
        ctx.query_host(0, 0, 0, log.S, host)
        np.testing.assert_array_equal(host, oracle.query(log, 0, 0, 0, log.S))
        # page-locked host memory: the scatter writes it directly
        pinned = torch.empty((log.S, log.V), dtype=torch.int32, pin_memory=True)
        for t in (1, 2):
            ctx.query_host(t, 3, 1, log.S - 1, pinned[: log.S - 1].numpy())
            np.testing.assert_array_equal(pinned[: log.S - 1].numpy().view(np.uint32),
                                          oracle.query(log, t, 3, 1, log.S - 1))


def test_error_paths(svv, small):
    log, ctx = small
    out = ctx.empty_out(8)
    for args in [(4, 0, 0, 1), (0, log.V, 0, 1), (0, 0, 0, 0), (0, 0, 5, 4)]:
        with pytest.raises(svv.SvvError) as e:
            svv.svv_query(ctx.h, *args, out)
        assert e.value.status == 1
    with svv.Context(0) as empty:
        with pytest.raises(svv.SvvError) as e:
            svv.svv_query(empty.h, 0, 0, 0, 1, out)
        assert e.value.status == 6
    # a round cap of 1 cannot finish: SVV_ETIMEOUT, and the context stays usable
    ctx.set_tuning("max_iters", 1)
    try:
        with pytest.raises(svv.SvvError) as e:
            ctx.query(0, 0, 0, 8)
        assert e.value.status == 4
    finally:
        ctx.set_tuning("max_iters", 0)
    np.testing.assert_array_equal(_iu(svv, ctx, 0, 0, 0, 8), oracle.query(log, 0, 0, 0, 8))
    with pytest.raises(svv.SvvError):
        ctx.set_tuning("no_such_key", 1)
    # a budget too small for the graph: SVV_ENOMEM
    with svv.Context(0, hbm_budget_bytes=4096) as tiny:
        with pytest.raises(svv.SvvError) as e:
            tiny.load_log(log)
        assert e.value.status == 2


@pytest.fixture(scope="module")
def rmat20(svv):
    log = W.rmat20()
    ctx = svv.Context(0)
    ctx.load_log(log)
    yield log, ctx
    ctx.close()


@pytest.mark.parametrize("t", [0, 1])
def test_rmat20_full(svv, rmat20, t):
    """RMAT scale 20, 64 snapshots, SSSP and SSWP from the top hub: every value."""
    log, ctx = rmat20
    q = W.rmat20_queries(log)[t]
    want = oracle.query(log, q.type, q.source, q.win_begin, q.win_len)
    np.testing.assert_array_equal(_iu(svv, ctx, q.type, q.source, q.win_begin, q.win_len), want)
    np.testing.assert_array_equal(_plain(svv, ctx, q.type, q.source, q.win_begin, q.win_len), want)
    cap, cup, row = ctx.bounds()
    ocap, ocup = oracle.bounds(log, q.type, q.source, q.win_begin, q.win_len)
    np.testing.assert_array_equal(cap, ocap)
    np.testing.assert_array_equal(cup, ocup)
