"""Stream-ordered queries (svv_query_async / svv_query_wait) and the bounded
device waits.

* Queries queued back to back, on one stream or alternating between two, give
  the oracle's values; a synchronous call after them is ordered after them; a
  ticket expires after 64 later queries.
* Failure detection without a fault: with the test hook "test_skip_arrival"
  one CTA of the intersection-graph solve leaves before its first barrier
  arrival, so the other CTAs' bounded waits (spin_limit_ms) expire; the query
  reports SVV_ETIMEOUT, synchronously and through svv_query_wait, and the next
  clean query on the same context matches the oracle.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__ as g
    g.build()
    from paper_2502_10579_gb300 import svv
    log = W.scaled_rmat(scale=13, edge_factor=8, n_snapshots=40, rate=0.003, seed=81)
    ctx = svv.Context(0)
    ctx.load_log(log)
    yield svv, log, ctx
    ctx.close()


def _specs(log, n, seed):
    rng = np.random.default_rng(seed)
    deg = np.bincount(log.src.astype(np.int64), minlength=log.V)
    hubs = np.argsort(-deg, kind="stable")[:8]
    out = []
    for k in range(n):
        L = int(rng.integers(1, log.S + 1))
        out.append((k % 4, int(hubs[k % len(hubs)]), int(rng.integers(0, log.S - L + 1)), L))
    return out


def test_async_one_stream(env):
    svv, log, ctx = env
    specs = _specs(log, 12, 1)
    outs = [ctx.empty_out(L) for (_, _, _, L) in specs]
    s = torch.cuda.Stream()
    tickets = [svv.svv_query_async(ctx.h, t, src, b, L, o, stream=s) for (t, src, b, L), o in zip(specs, outs)]
    for tk in tickets:
        assert svv.svv_query_wait(ctx.h, tk) == 0
    for (t, src, b, L), o in zip(specs, outs):
        np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, src, b, L))


def test_async_two_streams_then_sync(env):
    svv, log, ctx = env
    specs = _specs(log, 10, 2)
    outs = [ctx.empty_out(L) for (_, _, _, L) in specs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    tickets = [svv.svv_query_async(ctx.h, t, src, b, L, o, stream=streams[k % 2])
               for k, ((t, src, b, L), o) in enumerate(zip(specs, outs))]
    # a synchronous query on a third stream is ordered after the queued ones
    t, src, b, L = specs[3]
    mid = ctx.query(t, src, b, L, stream=torch.cuda.Stream())
    np.testing.assert_array_equal(svv.to_u32(mid), oracle.query(log, t, src, b, L))
    assert svv.svv_query_wait(ctx.h, tickets[-1], wait=True) == 0
    for tk in tickets:
        assert svv.svv_query_wait(ctx.h, tk, wait=False) == 0  # all done by now
    for (t, src, b, L), o in zip(specs, outs):
        np.testing.assert_array_equal(svv.to_u32(o), oracle.query(log, t, src, b, L))


def test_async_ticket_ring(env):
    svv, log, ctx = env
    out = ctx.empty_out(4)
    first = svv.svv_query_async(ctx.h, 2, 0, 0, 4, out)
    last = first
    for _ in range(70):
        last = svv.svv_query_async(ctx.h, 2, 0, 0, 4, out)
    assert svv.svv_query_wait(ctx.h, last) == 0
    with pytest.raises(svv.SvvError) as e:
        svv.svv_query_wait(ctx.h, first)
    assert e.value.status == 1
    with pytest.raises(svv.SvvError):
        svv.svv_query_wait(ctx.h, last + 1)  # never issued
    np.testing.assert_array_equal(svv.to_u32(out), oracle.query(log, 2, 0, 0, 4))


def test_bounded_wait_expires(env):
    svv, log, ctx = env
    deg = np.bincount(log.src.astype(np.int64), minlength=log.V)
    hub = int(np.argmax(deg))
    try:
        ctx.set_tuning("spin_limit_ms", 5)
        ctx.set_tuning("test_skip_arrival", 2)  # CTA 1 never arrives
        with pytest.raises(svv.SvvError) as e:
            ctx.query(0, hub, 0, log.S)
        assert e.value.status == 4  # SVV_ETIMEOUT
        out = ctx.empty_out(log.S)
        tk = svv.svv_query_async(ctx.h, 1, hub, 0, log.S, out)
        with pytest.raises(svv.SvvError) as e:
            svv.svv_query_wait(ctx.h, tk)
        assert e.value.status == 4
    finally:
        ctx.set_tuning("test_skip_arrival", 0)
        ctx.set_tuning("spin_limit_ms", 1000)
    # the context is usable right after
    for t in (0, 1, 2):
        np.testing.assert_array_equal(svv.to_u32(ctx.query(t, hub, 3, 20)), oracle.query(log, t, hub, 3, 20))
