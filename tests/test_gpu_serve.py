"""Serving: requests submitted while others run must each give exactly the
result of the same query run alone (and of the oracle), and the server must
overlap requests on the GPU and refuse work when its output arena is full."""
import time

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


def _requests(log, n, seed, l_hi):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = int(rng.integers(1, l_hi + 1))
        out.append((int(rng.integers(0, 4)), int(rng.integers(0, log.V)), int(rng.integers(0, log.S - L + 1)), L))
    return out


def test_serve_mix_equals_alone(svv):
    log = W.scaled_rmat(scale=14, edge_factor=8, n_snapshots=100, rate=0.002, seed=55, add_mode="skewed")
    reqs = _requests(log, 48, 9, 100)
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        alone = [svv.to_u32(ctx.query(t, s, b, L)) for t, s, b, L in reqs]
        svv.svv_serve_start(ctx.h, max_window=100, capacity=64)
        rng = np.random.default_rng(1)
        tickets = []
        for r in reqs:
            while True:
                tk = svv.svv_submit(ctx.h, *r)
                if tk is not None:
                    break
                time.sleep(0.001)  # arena full: admission waits for memory
            tickets.append(tk)
            time.sleep(float(rng.exponential(0.0005)))
        spans = []
        for tk, (t, s, b, L), want in zip(tickets, reqs, alone):
            assert svv.svv_poll(ctx.h, tk, wait=True) == 0
            addr, t0, t1 = svv.svv_ticket_info(ctx.h, tk)
            got = svv.device_u32(addr, L * log.V).reshape(L, log.V)
            np.testing.assert_array_equal(got, want)
            spans.append((t0, t1))
            svv.svv_release(ctx.h, tk)
        # requests overlapped on the device
        spans.sort()
        assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))
        for (t, s, b, L), want in list(zip(reqs, alone))[:2]:
            np.testing.assert_array_equal(want, oracle.query(log, t, s, b, L))
        svv.svv_serve_stop(ctx.h)


def test_serve_admission_and_relaunch(svv):
    log = W.small_rmat()
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        one = 8 * log.V * 4
        svv.svv_serve_start(ctx.h, max_window=8, capacity=16, arena_bytes=3 * one)
        tks = [svv.svv_submit(ctx.h, 0, 0, 0, 8) for _ in range(3)]
        assert all(t is not None for t in tks)
        assert svv.svv_submit(ctx.h, 0, 0, 0, 8) is None  # arena full: refused
        want = oracle.query(log, 0, 0, 0, 8)
        for tk in tks:
            assert svv.svv_poll(ctx.h, tk, wait=True) == 0
            addr, _, _ = svv.svv_ticket_info(ctx.h, tk)
            np.testing.assert_array_equal(svv.device_u32(addr, 8 * log.V).reshape(8, log.V), want)
            svv.svv_release(ctx.h, tk)
        # caller-owned output; after an idle period the server is relaunched
        time.sleep(0.5)
        out = ctx.empty_out(5)
        tk = svv.svv_submit(ctx.h, 2, 7, 3, 5, out=out)
        assert svv.svv_poll(ctx.h, tk, wait=True) == 0
        np.testing.assert_array_equal(svv.to_u32(out), oracle.query(log, 2, 7, 3, 5))
        svv.svv_release(ctx.h, tk)
        with pytest.raises(svv.SvvError):
            svv.svv_submit(ctx.h, 0, 0, 0, 9)  # longer than max_window
        svv.svv_serve_stop(ctx.h)


@pytest.mark.parametrize("gmax,mix", [(8, 0), (1, 0), (8, 1)])
def test_serve_groups(svv, gmax, mix):
    """batch_mode 2 (the mode of graphs from 2M vertices): a scheduler queues
    the submitted requests in query groups of up to group_max same-type
    requests, formed each time the previous group has its bounds.  Requests
    submitted while a group runs share the next group's rounds (their device
    spans overlap); with group_max 1 they run one after another.  A query on
    another stream in between is ordered with them, every result equals the
    query alone, and admission still refuses a full arena."""
    log = W.scaled_rmat(scale=13, edge_factor=8, n_snapshots=100, rate=0.003, seed=56, add_mode="skewed")
    deg = np.bincount(log.src.astype(np.int64), minlength=log.V)
    has_edges = np.flatnonzero(deg > 0)
    # sources with out-edges (an isolated source is answered alone, by a fill),
    # plus one isolated source
    reqs = [(t, int(has_edges[s % has_edges.size]), b, L) for t, s, b, L in _requests(log, 23, 11, 100)]
    reqs.insert(7, (0, int(np.flatnonzero(deg == 0)[0]), 5, 40))
    with svv.Context(0) as ctx:
        ctx.load_log(log)
        alone = [svv.to_u32(ctx.query(t, s, b, L)) for t, s, b, L in reqs]
        ctx.set_tuning("batch_mode", 2)
        ctx.set_tuning("group_max", gmax)
        ctx.set_tuning("group_mix", mix)
        svv.svv_serve_start(ctx.h, max_window=100, capacity=64, arena_bytes=900 * log.V * 4)
        side = torch.cuda.Stream()
        pending, spans, refused = [], [], 0

        def finish_oldest():
            tk, want = pending.pop(0)
            assert svv.svv_poll(ctx.h, tk, wait=True) == 0
            addr, t0, t1 = svv.svv_ticket_info(ctx.h, tk)
            L = want.shape[0]
            np.testing.assert_array_equal(svv.device_u32(addr, L * log.V).reshape(L, log.V), want)
            spans.append((t0, t1))
            svv.svv_release(ctx.h, tk)

        for k, (r, want) in enumerate(zip(reqs, alone)):
            tk = svv.svv_submit(ctx.h, *r)
            while tk is None:  # arena full: finish the oldest, then retry
                refused += 1
                finish_oldest()
                tk = svv.svv_submit(ctx.h, *r)
            pending.append((tk, want))
            if k == 4:  # a query on another stream while requests are queued
                t, s, b, L = reqs[0]
                mid = ctx.query(t, s, b, L, stream=side)
        side.synchronize()
        np.testing.assert_array_equal(svv.to_u32(mid), alone[0])
        while pending:
            finish_oldest()
        assert refused > 0
        assert all(t0 < t1 for t0, t1 in spans)
        order = sorted(spans)
        overlap = any(order[i + 1][0] < order[i][1] for i in range(len(order) - 1))
        assert overlap == (gmax > 1)  # shared rounds, or one after another
        svv.svv_serve_stop(ctx.h)
        t, s, b, L = reqs[1]
        np.testing.assert_array_equal(alone[1], oracle.query(log, t, s, b, L))
