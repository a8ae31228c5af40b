"""svv_solve_snapshot_noalloc: the entry point for callers that cannot allocate
device memory when they call (allocator-restricted code, plug-ins whose host
owns all memory, services that reserve memory up front).

It keeps its working memory in a fixed device array inside the library, so
this test checks, through the C ABI, that calls in a row give exactly the
values of the existing per-snapshot entry point (svv_query_plain) and of the
CPU oracle, and that a graph too large for the fixed array, an unsupported
query type and malformed CSRs are refused with SVV_EINVAL.  The file is named to be
collected last, and it builds everything it needs itself, so it passes alone
in a fresh process as well as after the other tests.
"""
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
    torch.cuda.set_device(0)
    return mod


def _device_csr(svv, log):
    rp, col, w, mask = svv.svv_build_versioned_csr(log.V, log.S, log.src, log.dst, log.w, log.t_add, log.t_del)
    dev = [torch.from_numpy(rp.view(np.int64)).cuda(), torch.from_numpy(col.view(np.int32)).cuda(),
           torch.from_numpy(w.view(np.int32)).cuda(), torch.from_numpy(mask.view(np.int64)).cuda()]
    return (rp, col, w, mask), dev


@pytest.mark.parametrize("make_log", [W.small_rmat, lambda: W.scaled_rmat(14, 8, 100, 0.002, 77, "skewed")])
def test_noalloc_matches_plain_twice(svv, make_log):
    log = make_log()
    host, dev = _device_csr(svv, log)
    E = int(host[1].shape[0])
    src = W.max_out_degree_vertex(log)
    with svv.Context(0) as ctx:
        ctx.load_csr(log.V, log.S, *host)
        calls = [(0, 0), (1, log.S - 1), (2, log.S // 2)]  # (type, snapshot)
        for qtype, snap in calls:  # consecutive calls share the fixed working memory
            want = svv.to_u32(ctx.query(qtype, src, snap, 1, plain=True))[0]
            np.testing.assert_array_equal(want, oracle.query(log, qtype, src, snap, 1)[0])
            out = torch.full((log.V,), -7, dtype=torch.int32, device="cuda:0")
            svv.svv_solve_snapshot_noalloc(qtype, log.V, E, log.S, *dev, snap, src, out)
            np.testing.assert_array_equal(svv.to_u32(out), want)


def test_noalloc_rejects_oversized_graph(svv):
    one = torch.zeros(4, dtype=torch.int64, device="cuda:0")
    out = torch.zeros(4, dtype=torch.int32, device="cuda:0")
    V = 3_000_000  # 4*V + 16*(V + E/64 + 64) is beyond the fixed 32 MiB
    with pytest.raises(svv.SvvError) as e:
        svv.svv_solve_snapshot_noalloc(0, V, 0, 1, one, one, one, one, 0, 0, out)
    assert e.value.status == 1


def _tiny(rp, col):
    """A 4-vertex graph on the device, every edge present in snapshot 0."""
    E = len(col)
    dev = [torch.tensor(rp, dtype=torch.int64, device="cuda:0"),
           torch.tensor(col + [0], dtype=torch.int32, device="cuda:0"),
           torch.ones(E + 1, dtype=torch.int32, device="cuda:0"),
           torch.full((E + 1,), 1, dtype=torch.int64, device="cuda:0")]
    return E, dev


def test_noalloc_rejects_ssnp(svv):
    E, dev = _tiny([0, 1, 2, 2, 2], [1, 2])
    out = torch.zeros(4, dtype=torch.int32, device="cuda:0")
    with pytest.raises(svv.SvvError) as e:
        svv.svv_solve_snapshot_noalloc(3, 4, E, 1, *dev, 0, 0, out)
    assert e.value.status == 1


@pytest.mark.parametrize("rp,col", [
    ([0, 1, 2, 2, 2], [1, 7]),      # a target >= V, reached in the second round
    ([0, 2, 1, 3, 3], [1, 2, 3]),   # a row that goes backwards
    ([0, 1, 2, 2, 2], [1, 2, 3]),   # row_ptr[V] != E
])
def test_noalloc_rejects_malformed_csr(svv, rp, col):
    """Inputs the kernel checks before it uses them: no access leaves the arrays."""
    E, dev = _tiny(rp, col)
    out = torch.zeros(4, dtype=torch.int32, device="cuda:0")
    with pytest.raises(svv.SvvError) as e:
        svv.svv_solve_snapshot_noalloc(0, 4, E, 1, *dev, 0, 0, out)
    assert e.value.status == 1
    # the fixed working memory is usable again right after a refused call
    E, dev = _tiny([0, 1, 2, 3, 3], [1, 2, 3])
    svv.svv_solve_snapshot_noalloc(2, 4, E, 1, *dev, 0, 0, out)
    assert svv.to_u32(out).tolist() == [0, 1, 2, 3]
