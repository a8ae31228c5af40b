"""Thin ctypes binding of libsvv's C ABI (include/svv.h).

Functions keep the C names and only marshal arguments: every step of a query
runs in the library's CUDA kernels.  Importing this module never falls back to
anything: if ``libsvv.so`` is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

SVV_SSSP, SVV_SSWP, SVV_BFS, SVV_SSNP = 0, 1, 2, 3
STATUS = {0: "SVV_OK", 1: "SVV_EINVAL", 2: "SVV_ENOMEM", 3: "SVV_ECUDA", 4: "SVV_ETIMEOUT",
          5: "SVV_EBUSY", 6: "SVV_ENOTLOADED", 7: "SVV_EINTERNAL"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsvv.so")

# every symbol include/svv.h declares
EXPORTS = ("svv_create", "svv_build_versioned_csr", "svv_load", "svv_query", "svv_query_plain",
           "svv_query_host", "svv_get_bounds", "svv_set_tuning", "svv_get_stats", "svv_device_bytes", "svv_status_str",
           "svv_last_error", "svv_destroy", "svv_solve_snapshot_noalloc",
           "svv_get_round_trace", "svv_query_batch", "svv_serve_start", "svv_submit", "svv_poll",
           "svv_ticket_info", "svv_release", "svv_serve_stop", "svv_serve_replay", "svv_autotune",
           "svv_query_compact", "svv_query_async", "svv_query_wait")


class SvvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class svv_query_spec(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("source", ctypes.c_uint32), ("win_begin", ctypes.c_uint32),
                ("win_len", ctypes.c_uint32), ("out", ctypes.c_void_p), ("status", ctypes.c_int)]


class svv_tune_result(ctypes.Structure):
    _fields_ = [("solve_chunk", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("relax_lanes", ctypes.c_uint32), ("skip_same", ctypes.c_uint32),
                ("pull_pct", ctypes.c_uint32), ("delta", ctypes.c_uint32), ("slab_max", ctypes.c_uint32),
                ("best_ms", ctypes.c_float), ("default_ms", ctypes.c_float), ("candidates", ctypes.c_uint32)]


class svv_stats(ctypes.Structure):
    _fields_ = [("unstable", ctypes.c_uint32), ("qrs_edges", ctypes.c_uint32),
                ("qrs_masked", ctypes.c_uint32), ("iters_cap", ctypes.c_uint32),
                ("iters_cup", ctypes.c_uint32), ("iters_relax", ctypes.c_uint32),
                ("iters_plain_max", ctypes.c_uint32), ("phase_timing", ctypes.c_uint32),
                ("edges_relaxed_cap", ctypes.c_uint64), ("edges_relaxed_cup", ctypes.c_uint64),
                ("edges_relaxed_multi", ctypes.c_uint64), ("ms_cap", ctypes.c_float),
                ("ms_cup", ctypes.c_float), ("ms_qrs", ctypes.c_float), ("ms_relax", ctypes.c_float),
                ("ms_scatter", ctypes.c_float), ("ms_batch", ctypes.c_float),
                ("batch_teams", ctypes.c_uint32), ("batch_team_blocks", ctypes.c_uint32),
                ("ms_group_cap", ctypes.c_float), ("ms_group_cup", ctypes.c_float)]


_lib = None


def lib():
    """Load libsvv.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P, u32, u64, i32, i64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_int64
    L.svv_create.argtypes = [ctypes.POINTER(P), i32, u64]
    L.svv_build_versioned_csr.argtypes = [u32, u32, u64, P, P, P, P, P, P, P, P, P, ctypes.POINTER(u64)]
    L.svv_load.argtypes = [P, u32, u64, u32, P, P, P, P, i32]
    q = [P, i32, u32, u32, u32, P, P]
    L.svv_query.argtypes = q
    L.svv_query_plain.argtypes = q
    L.svv_query_host.argtypes = q
    L.svv_get_bounds.argtypes = [P, P, P, P, P]
    L.svv_set_tuning.argtypes = [P, ctypes.c_char_p, i64]
    L.svv_get_stats.argtypes = [P, ctypes.POINTER(svv_stats)]
    L.svv_device_bytes.argtypes = [P]
    L.svv_device_bytes.restype = u64
    L.svv_status_str.argtypes = [i32]
    L.svv_status_str.restype = ctypes.c_char_p
    L.svv_last_error.argtypes = [P]
    L.svv_last_error.restype = ctypes.c_char_p
    L.svv_destroy.argtypes = [P]
    L.svv_destroy.restype = None
    L.svv_solve_snapshot_noalloc.argtypes = [i32, u32, u64, u32, P, P, P, P, u32, u32, P, P]
    L.svv_solve_snapshot_noalloc.restype = i32
    L.svv_get_round_trace.argtypes = [P, u32, P, u32, ctypes.POINTER(u32)]
    L.svv_get_round_trace.restype = i32
    L.svv_query_batch.argtypes = [P, u32, ctypes.POINTER(svv_query_spec), P]
    L.svv_query_batch.restype = i32
    L.svv_serve_start.argtypes = [P, u32, u32, u64]
    L.svv_submit.argtypes = [P, ctypes.POINTER(svv_query_spec), ctypes.POINTER(u64)]
    L.svv_poll.argtypes = [P, u64, i32, ctypes.POINTER(i32)]
    L.svv_ticket_info.argtypes = [P, u64, ctypes.POINTER(P), ctypes.POINTER(u64), ctypes.POINTER(u64)]
    L.svv_release.argtypes = [P, u64]
    L.svv_serve_stop.argtypes = [P]
    L.svv_serve_replay.argtypes = [P, u32, ctypes.POINTER(svv_query_spec), P, P, P]
    L.svv_autotune.argtypes = [P, i32, u32, u32, u32, u32, ctypes.POINTER(svv_tune_result)]
    L.svv_autotune.restype = i32
    L.svv_query_compact.argtypes = [P, i32, u32, u32, u32, P, P, P, u64, ctypes.POINTER(u32), P]
    L.svv_query_compact.restype = i32
    L.svv_query_async.argtypes = [P, i32, u32, u32, u32, P, P, ctypes.POINTER(u64)]
    L.svv_query_async.restype = i32
    L.svv_query_wait.argtypes = [P, u64, i32]
    L.svv_query_wait.restype = i32
    for f in ("svv_serve_start", "svv_submit", "svv_poll", "svv_ticket_info", "svv_release", "svv_serve_stop",
              "svv_serve_replay"):
        getattr(L, f).restype = i32
    for f in ("svv_create", "svv_build_versioned_csr", "svv_load", "svv_query", "svv_query_plain",
              "svv_query_host", "svv_get_bounds", "svv_set_tuning", "svv_get_stats"):
        getattr(L, f).restype = i32
    _lib = L
    return L


def _check(ctx, st: int):
    if st != 0:
        msg = lib().svv_last_error(ctx).decode() if ctx else ""
        raise SvvError(st, msg)


def _ptr(x):
    """Address of a numpy array or a torch tensor."""
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


def _stream(stream):
    if stream is None:
        try:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# --------------------------------------------------------------------------
# C-ABI mirrors
def svv_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = ctypes.c_void_p()
    _check(None, lib().svv_create(ctypes.byref(h), device, hbm_budget_bytes))
    return h


def svv_destroy(ctx):
    lib().svv_destroy(ctx)


def svv_status_str(st: int) -> str:
    return lib().svv_status_str(st).decode()


def svv_last_error(ctx) -> str:
    return lib().svv_last_error(ctx).decode()


def svv_device_bytes(ctx) -> int:
    return int(lib().svv_device_bytes(ctx))


def svv_set_tuning(ctx, key: str, value: int):
    _check(ctx, lib().svv_set_tuning(ctx, key.encode(), int(value)))


def svv_get_stats(ctx) -> dict:
    s = svv_stats()
    _check(ctx, lib().svv_get_stats(ctx, ctypes.byref(s)))
    return {name: (float(getattr(s, name)) if name.startswith("ms_") else int(getattr(s, name)))
            for name, _ in svv_stats._fields_ if name != "reserved"}


def svv_build_versioned_csr(V: int, S: int, src, dst, w, t_add, t_del):
    """Host builder: edge instances with live interval [t_add, t_del) ->
    (row_ptr u64[V+1], col u32[E], weight u32[E], mask u64[E*W])."""
    src = np.ascontiguousarray(src, np.uint32)
    dst = np.ascontiguousarray(dst, np.uint32)
    w = np.ascontiguousarray(w, np.uint32)
    t_add = np.ascontiguousarray(t_add, np.uint32)
    t_del = np.ascontiguousarray(t_del, np.uint32)
    n = src.shape[0]
    W = (S + 63) // 64
    row_ptr = np.empty(V + 1, np.uint64)
    col = np.empty(max(n, 1), np.uint32)
    weight = np.empty(max(n, 1), np.uint32)
    mask = np.empty(max(n, 1) * W, np.uint64)
    E = ctypes.c_uint64()
    _check(None, lib().svv_build_versioned_csr(V, S, n, _ptr(src), _ptr(dst), _ptr(w), _ptr(t_add),
                                               _ptr(t_del), _ptr(row_ptr), _ptr(col), _ptr(weight),
                                               _ptr(mask), ctypes.byref(E)))
    E = int(E.value)
    return row_ptr, col[:E], weight[:E], mask[:E * W]


def svv_load(ctx, V: int, E: int, S: int, row_ptr, col, weight, mask, inputs_on_device: bool = False):
    _check(ctx, lib().svv_load(ctx, V, E, S, _ptr(row_ptr), _ptr(col), _ptr(weight), _ptr(mask),
                               1 if inputs_on_device else 0))


def svv_query(ctx, qtype: int, source: int, win_begin: int, win_len: int, out, stream=None):
    _check(ctx, lib().svv_query(ctx, qtype, source, win_begin, win_len, _ptr(out), _stream(stream)))


def svv_query_async(ctx, qtype: int, source: int, win_begin: int, win_len: int, out, stream=None) -> int:
    """Queue a query on the stream and return its ticket (no host wait)."""
    t = ctypes.c_uint64()
    _check(ctx, lib().svv_query_async(ctx, qtype, source, win_begin, win_len, _ptr(out), _stream(stream),
                                      ctypes.byref(t)))
    return int(t.value)


def svv_query_wait(ctx, ticket: int, wait: bool = True):
    """The status of a queued query (raises on failure), or None while it runs (wait=False)."""
    st = lib().svv_query_wait(ctx, ticket, 1 if wait else 0)
    if st == 5:
        return None
    _check(ctx, st)
    return 0


def svv_query_plain(ctx, qtype: int, source: int, win_begin: int, win_len: int, out, stream=None):
    _check(ctx, lib().svv_query_plain(ctx, qtype, source, win_begin, win_len, _ptr(out), _stream(stream)))


def svv_query_host(ctx, qtype: int, source: int, win_begin: int, win_len: int, out_host, stream=None):
    _check(ctx, lib().svv_query_host(ctx, qtype, source, win_begin, win_len, _ptr(out_host),
                                     _stream(stream)))


def svv_query_batch(ctx, specs, stream=None):
    """specs: list of (type, source, win_begin, win_len, out_tensor).  Returns
    the per-instance statuses; raises on a batch-level failure only when no
    instance could run."""
    n = len(specs)
    arr = (svv_query_spec * max(n, 1))()
    for i, (t, s, b, L, out) in enumerate(specs):
        arr[i].type, arr[i].source, arr[i].win_begin, arr[i].win_len = t, s, b, L
        arr[i].out = _ptr(out).value if out is not None else None
        arr[i].status = -1
    st = lib().svv_query_batch(ctx, n, arr, _stream(stream))
    statuses = [int(arr[i].status) for i in range(n)]
    if st != 0 and all(x != 0 for x in statuses):
        _check(ctx, st)
    return statuses


def svv_query_compact(ctx, qtype: int, source: int, win_begin: int, win_len: int, cap_out, row_out, rows_out,
                      stream=None) -> int:
    """Compact result into device tensors; returns U (number of rows)."""
    u = ctypes.c_uint32()
    _check(ctx, lib().svv_query_compact(ctx, qtype, source, win_begin, win_len, _ptr(cap_out), _ptr(row_out),
                                        _ptr(rows_out), rows_out.numel(), ctypes.byref(u), _stream(stream)))
    return int(u.value)


def svv_autotune(ctx, qtype: int, source: int, win_begin: int, win_len: int, reps: int = 3) -> dict:
    r = svv_tune_result()
    _check(ctx, lib().svv_autotune(ctx, qtype, source, win_begin, win_len, reps, ctypes.byref(r)))
    return {name: (float(getattr(r, name)) if name.endswith("_ms") else int(getattr(r, name)))
            for name, _ in svv_tune_result._fields_}


def svv_serve_start(ctx, max_window: int, capacity: int = 4096, arena_bytes: int = 0):
    _check(ctx, lib().svv_serve_start(ctx, max_window, capacity, arena_bytes))


def svv_submit(ctx, qtype: int, source: int, win_begin: int, win_len: int, out=None):
    """Queue a request; returns its ticket, or None when the server is full (SVV_EBUSY)."""
    spec = svv_query_spec()
    spec.type, spec.source, spec.win_begin, spec.win_len = qtype, source, win_begin, win_len
    spec.out = _ptr(out).value if out is not None else None
    t = ctypes.c_uint64()
    st = lib().svv_submit(ctx, ctypes.byref(spec), ctypes.byref(t))
    if st == 5:
        return None
    _check(ctx, st)
    return int(t.value)


def svv_poll(ctx, ticket: int, wait: bool = False):
    """The request's status once done, else None."""
    r = ctypes.c_int()
    st = lib().svv_poll(ctx, ticket, 1 if wait else 0, ctypes.byref(r))
    if st == 5:
        return None
    _check(ctx, st)
    return int(r.value)


def svv_ticket_info(ctx, ticket: int):
    """(device output address, device start ns, device end ns)."""
    out, t0, t1 = ctypes.c_void_p(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(ctx, lib().svv_ticket_info(ctx, ticket, ctypes.byref(out), ctypes.byref(t0), ctypes.byref(t1)))
    return int(out.value or 0), int(t0.value), int(t1.value)


def svv_release(ctx, ticket: int):
    _check(ctx, lib().svv_release(ctx, ticket))


def svv_serve_replay(ctx, requests):
    """requests: list of (arrival_s, type, source, win_begin, win_len).  Returns
    (latency_ms, done_s) numpy arrays; outputs come from the server's arena."""
    n = len(requests)
    arr = (svv_query_spec * max(n, 1))()
    at = np.zeros(max(n, 1), np.float64)
    for i, (a, t, s, b, L) in enumerate(requests):
        arr[i].type, arr[i].source, arr[i].win_begin, arr[i].win_len, arr[i].out = t, s, b, L, None
        at[i] = a
    lat = np.zeros(max(n, 1), np.float64)
    done = np.zeros(max(n, 1), np.float64)
    _check(ctx, lib().svv_serve_replay(ctx, n, arr, _ptr(at), _ptr(lat), _ptr(done)))
    return lat[:n], done[:n]


def svv_serve_stop(ctx):
    _check(ctx, lib().svv_serve_stop(ctx))


_cudart = None


def device_u32(address: int, n: int) -> np.ndarray:
    """Copy n uint32 at a device address (e.g. a serving arena output) to host."""
    global _cudart
    if _cudart is None:
        for name in ("libcudart.so", "libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
            try:
                _cudart = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if _cudart is None:
            raise RuntimeError("libcudart not found")
        _cudart.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        _cudart.cudaMemcpy.restype = ctypes.c_int
    out = np.empty(n, np.uint32)
    if n:
        rc = _cudart.cudaMemcpy(out.ctypes.data, address, 4 * n, 2)  # cudaMemcpyDeviceToHost
        if rc != 0:
            raise RuntimeError(f"cudaMemcpy failed ({rc})")
    return out


def svv_get_round_trace(ctx, phase: int):
    """[(frontier_units, start_ns)] per round of the last query's phase
    (0 intersection, 1 union, 2 relaxation); round 0 holds (0, init_end_ns).
    Phase 3 (subgraph extraction): the six pass timestamps in ns."""
    buf = np.zeros(4096, np.uint64)
    n = ctypes.c_uint32()
    _check(ctx, lib().svv_get_round_trace(ctx, phase, _ptr(buf), 4096, ctypes.byref(n)))
    if phase == 3:
        return [int(x) for x in buf[:6]]
    out = []
    for i, x in enumerate(buf[:n.value].tolist()):
        if x == 0 and i > 0:
            break
        out.append((x >> 40, x & ((1 << 40) - 1)))
    return out


def svv_get_bounds(ctx, cap=None, cup=None, row=None, stream=None):
    n = ctypes.c_void_p(0)
    _check(ctx, lib().svv_get_bounds(ctx, _ptr(cap) if cap is not None else n,
                                     _ptr(cup) if cup is not None else n,
                                     _ptr(row) if row is not None else n, _stream(stream)))


def svv_solve_snapshot_noalloc(qtype: int, V: int, E: int, S: int, row_ptr, col, weight, mask,
                               snapshot: int, source: int, out, stream=None):
    """One snapshot's solve with no allocation; all arrays are device tensors."""
    _check(None, lib().svv_solve_snapshot_noalloc(qtype, V, E, S, _ptr(row_ptr), _ptr(col), _ptr(weight),
                                                  _ptr(mask), snapshot, source, _ptr(out), _stream(stream)))


# --------------------------------------------------------------------------
@dataclass
class LoadedGraph:
    V: int
    S: int
    E: int


class Context:
    """Owns one svv context; convenience over the C-ABI mirrors above."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.h = svv_create(device, hbm_budget_bytes)
        self.graph = None

    def close(self):
        if self.h is not None:
            svv_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_log(self, log) -> LoadedGraph:
        """Build the versioned union graph of an edge log and load it."""
        rp, col, w, mask = svv_build_versioned_csr(log.V, log.S, log.src, log.dst, log.w, log.t_add, log.t_del)
        return self.load_csr(log.V, log.S, rp, col, w, mask)

    def load_csr(self, V, S, row_ptr, col, weight, mask, inputs_on_device=False) -> LoadedGraph:
        E = int(col.shape[0])
        svv_load(self.h, V, E, S, row_ptr, col, weight, mask, inputs_on_device)
        self.graph = LoadedGraph(V, S, E)
        return self.graph

    def set_tuning(self, key, value):
        svv_set_tuning(self.h, key, value)

    def stats(self) -> dict:
        return svv_get_stats(self.h)

    def device_bytes(self) -> int:
        return svv_device_bytes(self.h)

    def empty_out(self, win_len: int):
        import torch
        return torch.empty((win_len, self.graph.V), dtype=torch.int32, device=f"cuda:{self.device}")

    def query(self, qtype, source, win_begin, win_len, out=None, stream=None, plain=False):
        """Run one query; returns the (win_len, V) int32 tensor holding uint32 values."""
        if out is None:
            out = self.empty_out(win_len)
        fn = svv_query_plain if plain else svv_query
        fn(self.h, qtype, source, win_begin, win_len, out, stream)
        return out

    def query_batch(self, specs, stream=None):
        """specs: list of (type, source, win_begin, win_len[, out]); returns
        (outputs, statuses)."""
        full = []
        for sp in specs:
            t, s, b, L = sp[:4]
            out = sp[4] if len(sp) > 4 else self.empty_out(L)
            full.append((t, s, b, L, out))
        st = svv_query_batch(self.h, full, stream)
        return [f[4] for f in full], st

    def bounds(self):
        """(intersection values, union values, row map) of the last query, as uint32 numpy."""
        import torch
        V = self.graph.V
        t = [torch.empty(V, dtype=torch.int32, device=f"cuda:{self.device}") for _ in range(3)]
        svv_get_bounds(self.h, *t)
        return tuple(to_u32(x) for x in t)

    def query_host(self, qtype, source, win_begin, win_len, out_host, stream=None):
        svv_query_host(self.h, qtype, source, win_begin, win_len, out_host, stream)
        return out_host


def to_u32(t) -> np.ndarray:
    """Copy a result tensor to host as uint32."""
    return t.cpu().numpy().view(np.uint32)
