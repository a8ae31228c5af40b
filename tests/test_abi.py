"""CPU-side checks of the C ABI: the library loads, exports every function the
header declares, and its host-only builder writes the Section 4.1 version
labels (bit i = snapshot i, least significant bit = snapshot 0)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def svv():
    import __graft_entry__ as g
    g.build()
    from paper_2502_10579_gb300 import svv as mod
    mod.lib()
    return mod


def _declared():
    with open(os.path.join(ROOT, "include", "svv.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(svv_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(svv):
    declared = _declared()
    assert len(declared) >= 12
    L = svv.lib()
    for name in declared:
        assert hasattr(L, name), f"libsvv.so does not export {name}"
    assert sorted(svv.EXPORTS) == declared


def test_status_strings(svv):
    for k, v in svv.STATUS.items():
        assert svv.svv_status_str(k) == v


def test_builder_version_labels(svv):
    # Section 4.1: an instance live in snapshots 0 and 3 only is two instances
    # under the instance model (deleted at 1, re-added at 3): labels 0b0001 and
    # 0b1000; an instance live in every snapshot is all ones (0b1111).
    V, S = 5, 4
    src = np.array([3, 3, 4, 0], np.uint32)  # D=3 -> C=2 twice, E=4 -> C=2, A=0 -> E=4
    dst = np.array([2, 2, 2, 4], np.uint32)
    w = np.array([1, 1, 2, 3], np.uint32)
    t_add = np.array([0, 3, 0, 0], np.uint32)
    t_del = np.array([1, 4, 4, 1], np.uint32)
    rp, col, wt, mask = svv.svv_build_versioned_csr(V, S, src, dst, w, t_add, t_del)
    assert rp.tolist() == [0, 1, 1, 1, 3, 4]
    assert mask.tolist() == [0b0001, 0b0001, 0b1000, 0b1111]
    assert col.tolist() == [4, 2, 2, 2]


def test_builder_two_words(svv):
    V, S = 3, 100
    src = np.array([0, 1, 2], np.uint32)
    dst = np.array([1, 2, 0], np.uint32)
    w = np.array([5, 6, 7], np.uint32)
    t_add = np.array([60, 0, 64], np.uint32)
    t_del = np.array([70, 100, 65], np.uint32)
    rp, col, wt, mask = svv.svv_build_versioned_csr(V, S, src, dst, w, t_add, t_del)
    m = mask.reshape(-1, 2)
    assert m[0].tolist() == [0xF << 60, (1 << 6) - 1]
    assert m[1].tolist() == [(1 << 64) - 1, (1 << 36) - 1]
    assert m[2].tolist() == [0, 1]


def test_builder_matches_log_intervals(svv):
    import workloads as W
    log = W.random_small_log(3, V=30, n_edges=90, S=70, n_add=5, n_del=4)
    rp, col, wt, mask = svv.svv_build_versioned_csr(log.V, log.S, log.src, log.dst, log.w, log.t_add, log.t_del)
    m = mask.reshape(-1, 2)
    rows = np.repeat(np.arange(log.V), np.diff(rp.astype(np.int64)))
    order = np.argsort(log.src, kind="stable")
    assert (rows == log.src[order]).all() and (col == log.dst[order]).all() and (wt == log.w[order]).all()
    for e, k in enumerate(order):
        for i in range(log.S):
            live = log.t_add[k] <= i < log.t_del[k]
            assert bool((int(m[e, i // 64]) >> (i % 64)) & 1) == live


def test_builder_rejects_bad_input(svv):
    one = np.zeros(1, np.uint32)
    with pytest.raises(svv.SvvError):
        svv.svv_build_versioned_csr(4, 0, one, one, one, one, one)
    with pytest.raises(svv.SvvError):
        svv.svv_build_versioned_csr(4, 8, np.array([9], np.uint32), one, one, one, one)
    with pytest.raises(svv.SvvError):
        svv.svv_build_versioned_csr(4, 8, one, one, one, one, np.array([9], np.uint32))
