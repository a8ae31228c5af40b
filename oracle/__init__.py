"""CPU oracle for stable-vertex-value queries -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
use this package.  The library under ``paper_2502_10579_gb300`` never imports
it, and it imports nothing from the library.

``oracle.c`` solves each snapshot of a window from scratch on the snapshot
materialised by replaying the edge log (paper Section 2, Fig. 2a): binary-heap
Dijkstra for SSSP, widest-path Dijkstra for SSWP, a FIFO BFS and narrowest-path
Dijkstra for SSNP (Table 2).
``bounds()`` solves the intersection and union graphs of a window (Section 3,
Step 1).  ``live_intervals()`` and ``window_csr()`` give the same graphs (and
every snapshot, as a one-snapshot window) from one replay of the log, for
checks over many windows.  Value encoding: SSSP/BFS/SSNP unreachable =
0xFFFFFFFF; SSWP source = 0xFFFFFFFF (+inf) and unreachable = 0; SSSP sums
saturate at 0xFFFFFFFE.

Every function is pinned by ``tests/test_oracle_pins.py`` (Floyd-Warshall
brute force, SciPy's graph routines, a pure-Python replay, Theorems 1 and 2,
and the hand-solved fixtures under ``tests/golden/``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

SSSP, SSWP, BFS, SSNP = 0, 1, 2, 3
INF = 0xFFFFFFFF

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (portable flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC",
                               "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
            lib.oracle_solve.argtypes = [i32, u32, P, P, P, u32, P]
            lib.oracle_query.argtypes = [i32, u32, u32, u64, P, P, P, P, P, P, u32, u32, u32, P, i32]
            lib.oracle_bounds.argtypes = [i32, u32, u32, u64, P, P, P, P, P, P, u32, u32, u32, P, P]
            lib.oracle_snapshot_csr.argtypes = [u32, u32, u64, P, P, P, P, P, P, u32, P,
                                                ctypes.POINTER(P), ctypes.POINTER(P)]
            lib.oracle_free.argtypes = [P]
            lib.oracle_live_intervals.argtypes = [u32, u32, u64, P, P, P, P, P, P, P, P]
            lib.oracle_window_csr.argtypes = [u32, u32, u64, P, P, P, P, P, u32, u32, i32, P,
                                              ctypes.POINTER(P), ctypes.POINTER(P)]
            for f in (lib.oracle_solve, lib.oracle_query, lib.oracle_bounds, lib.oracle_snapshot_csr,
                      lib.oracle_live_intervals, lib.oracle_window_csr):
                f.restype = i32
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc == -1:
        raise MemoryError(f"oracle {what}: out of memory")
    if rc != 0:
        raise ValueError(f"oracle {what}: bad arguments (rc={rc})")


def _log_arrays(log):
    return (np.ascontiguousarray(log.src, np.uint32), np.ascontiguousarray(log.dst, np.uint32),
            np.ascontiguousarray(log.w, np.uint32), np.ascontiguousarray(log.add_off, np.int64),
            np.ascontiguousarray(log.del_off, np.int64), np.ascontiguousarray(log.del_ids, np.int64))


def solve(qtype: int, V: int, row_ptr, col, w, source: int) -> np.ndarray:
    """Single-source solve of one query type on one CSR graph (Table 2)."""
    rp = np.ascontiguousarray(row_ptr, np.uint64)
    c = np.ascontiguousarray(col, np.uint32)
    ww = np.ascontiguousarray(w, np.uint32)
    out = np.empty(V, np.uint32)
    _check(_L().oracle_solve(qtype, V, _p(rp), _p(c), _p(ww), source, _p(out)), "solve")
    return out


def query(log, qtype: int, source: int, win_begin: int, win_len: int, nthreads: int = 0) -> np.ndarray:
    """``out[i, v]`` = value of ``v`` in snapshot ``win_begin + i`` (shape ``(win_len, V)``)."""
    a = _log_arrays(log)
    out = np.empty((win_len, log.V), np.uint32)
    rc = _L().oracle_query(qtype, log.V, log.S, a[0].shape[0], *[_p(x) for x in a], source,
                           win_begin, win_len, _p(out), nthreads)
    _check(rc, "query")
    return out


def bounds(log, qtype: int, source: int, win_begin: int, win_len: int):
    """(values on the window's intersection graph, values on its union graph)."""
    a = _log_arrays(log)
    cap = np.empty(log.V, np.uint32)
    cup = np.empty(log.V, np.uint32)
    rc = _L().oracle_bounds(qtype, log.V, log.S, a[0].shape[0], *[_p(x) for x in a], source,
                            win_begin, win_len, _p(cap), _p(cup))
    _check(rc, "bounds")
    return cap, cup


def snapshot_csr(log, snap: int):
    """CSR ``(row_ptr, col, w)`` of snapshot ``snap``, materialised by replay."""
    a = _log_arrays(log)
    rp = np.empty(log.V + 1, np.uint64)
    cp, wp = ctypes.c_void_p(), ctypes.c_void_p()
    rc = _L().oracle_snapshot_csr(log.V, log.S, a[0].shape[0], *[_p(x) for x in a], snap, _p(rp),
                                  ctypes.byref(cp), ctypes.byref(wp))
    _check(rc, "snapshot_csr")
    m = int(rp[-1])
    try:
        col = np.ctypeslib.as_array(ctypes.cast(cp, ctypes.POINTER(ctypes.c_uint32)), (max(m, 1),))[:m].copy()
        w = np.ctypeslib.as_array(ctypes.cast(wp, ctypes.POINTER(ctypes.c_uint32)), (max(m, 1),))[:m].copy()
    finally:
        _L().oracle_free(cp)
        _L().oracle_free(wp)
    return rp, col, w


def live_intervals(log):
    """(t_add, t_del): instance k is live exactly in snapshots [t_add[k], t_del[k]),
    from one replay of the log's steps (Section 2)."""
    a = _log_arrays(log)
    n = a[0].shape[0]
    t_add = np.empty(max(n, 1), np.uint32)
    t_del = np.empty(max(n, 1), np.uint32)
    _check(_L().oracle_live_intervals(log.V, log.S, n, *[_p(x) for x in a], _p(t_add), _p(t_del)), "live_intervals")
    return t_add[:n], t_del[:n]


def window_csr(log, intervals, win_begin: int, win_len: int, kind: str):
    """CSR ``(row_ptr, col, w)`` of the window's intersection graph
    (``kind="cap"``: instances live in every window snapshot) or union graph
    (``kind="cup"``: live in at least one), Section 3 Step 1; a one-snapshot
    window is that snapshot."""
    a = _log_arrays(log)
    t_add, t_del = (np.ascontiguousarray(x, np.uint32) for x in intervals)
    rp = np.empty(log.V + 1, np.uint64)
    cp, wp = ctypes.c_void_p(), ctypes.c_void_p()
    rc = _L().oracle_window_csr(log.V, log.S, a[0].shape[0], _p(a[0]), _p(a[1]), _p(a[2]), _p(t_add), _p(t_del),
                                win_begin, win_len, {"cap": 0, "cup": 1}[kind], _p(rp), ctypes.byref(cp),
                                ctypes.byref(wp))
    _check(rc, "window_csr")
    m = int(rp[-1])
    try:
        col = np.ctypeslib.as_array(ctypes.cast(cp, ctypes.POINTER(ctypes.c_uint32)), (max(m, 1),))[:m].copy()
        w = np.ctypeslib.as_array(ctypes.cast(wp, ctypes.POINTER(ctypes.c_uint32)), (max(m, 1),))[:m].copy()
    finally:
        _L().oracle_free(cp)
        _L().oracle_free(wp)
    return rp, col, w
