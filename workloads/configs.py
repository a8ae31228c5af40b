"""The five synthetic workloads (and scaled-down copies of them for tests).

Each preset returns an ``EdgeLog`` plus the queries run on it.  Sizes, weight
ranges, delta rates and query mixes follow the workloads the library is
measured on; seeds are ``1000 + workload number``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .rmat import EdgeLog, make_log, max_out_degree_vertex

SSSP, SSWP, BFS, SSNP = 0, 1, 2, 3
TYPE_NAMES = {SSSP: "sssp", SSWP: "sswp", BFS: "bfs", SSNP: "ssnp"}


@dataclass
class Query:
    type: int
    source: int
    win_begin: int
    win_len: int


def small_rmat(seed: int = 1001) -> EdgeLog:
    """RMAT, 4,096 vertices, 32,768 edges, w in [1,255], 8 snapshots; each step
    deletes 1% (328) of the live instances and adds 328 uniform-endpoint ones."""
    return make_log(scale=12, n_edges=32768, n_snapshots=8, n_add=328, n_del=328,
                    w_lo=1, w_hi=255, seed=seed, add_mode="uniform")


def rmat20(seed: int = 1002, n_snapshots: int = 64) -> EdgeLog:
    """RMAT scale 20 (1,048,576 vertices, 16,777,216 edges), w in [1,999],
    64 snapshots; each step deletes 10,000 uniform live instances and adds
    10,000 RMAT-distributed ones."""
    return make_log(scale=20, n_edges=1 << 24, n_snapshots=n_snapshots, n_add=10000,
                    n_del=10000, w_lo=1, w_hi=999, seed=seed, add_mode="rmat")


def rmat22(seed: int = 1003, n_snapshots: int = 64) -> EdgeLog:
    """RMAT scale 22 (4,194,304 vertices, 67,108,864 edges), w in [1,999];
    per step 0.05% of the edges change: 16,777 RMAT additions and 16,777
    uniform deletions."""
    d = round(0.0005 * (1 << 26))
    add = d // 2
    return make_log(scale=22, n_edges=1 << 26, n_snapshots=n_snapshots, n_add=add,
                    n_del=d - add, w_lo=1, w_hi=999, seed=seed, add_mode="rmat")


def rmat24(seed: int = 1004) -> EdgeLog:
    """RMAT scale 24 (16,777,216 vertices, 268,435,456 edges), w in [1,999],
    100 snapshots (two presence words); per step 0.1% of the edges change,
    additions with degree-skewed endpoints."""
    d = round(0.001 * (1 << 28))
    add = d // 2
    return make_log(scale=24, n_edges=1 << 28, n_snapshots=100, n_add=add, n_del=d - add,
                    w_lo=1, w_hi=999, seed=seed, add_mode="skewed")


def scaled_rmat(scale: int, edge_factor: int, n_snapshots: int, rate: float, seed: int,
                add_mode: str = "rmat", w_hi: int = 999) -> EdgeLog:
    """A smaller copy of the large workloads with the same shape."""
    E = edge_factor << scale
    d = max(2, round(rate * E))
    add = d // 2
    return make_log(scale=scale, n_edges=E, n_snapshots=n_snapshots, n_add=add,
                    n_del=d - add, w_lo=1, w_hi=w_hi, seed=seed, add_mode=add_mode)


def rmat20_queries(log: EdgeLog):
    """SSSP and SSWP from the highest-out-degree vertex of G_0, window [0, 64)."""
    s = max_out_degree_vertex(log)
    return [Query(SSSP, s, 0, log.S), Query(SSWP, s, 0, log.S)]


def batch_queries(log: EdgeLog, n: int = 256, seed: int = 3, l_lo: int = 8, l_hi: int = 64):
    """A mixed batch: 1/3 each of SSSP/SSWP/BFS in shuffled order, uniform
    sources, window length uniform in [l_lo, l_hi] at a uniform offset."""
    rng = np.random.default_rng(seed)
    types = np.array([SSSP] * ((n + 2) // 3) + [SSWP] * ((n + 1) // 3) + [BFS] * (n // 3))
    types = types[np.argsort(rng.random(n), kind="stable")]
    l_hi = min(l_hi, log.S)
    l_lo = min(l_lo, l_hi)
    out = []
    for t in types:
        src = int(rng.integers(0, log.V))
        L = int(rng.integers(l_lo, l_hi + 1))
        b = int(rng.integers(0, log.S - L + 1))
        out.append(Query(int(t), src, b, L))
    return out


def rmat24_queries(log: EdgeLog, n_sources: int = 16, seed: int = 4, windows=(25, 50, 100)):
    """SSSP and BFS from n_sources sources (uniform among vertices with
    out-degree > 0 in G_0) over the windows [0, L): 2 * n_sources * len(windows)
    queries, run one at a time."""
    rng = np.random.default_rng(seed)
    deg = np.bincount(log.src[: log.n_base].astype(np.int64), minlength=log.V)
    cand = np.flatnonzero(deg > 0)
    srcs = cand[rng.integers(0, cand.shape[0], size=n_sources)]
    out = []
    for s in srcs.tolist():
        for L in windows:
            L = min(L, log.S)
            out.append(Query(SSSP, int(s), 0, L))
            out.append(Query(BFS, int(s), 0, L))
    return out


def serve_requests(log: EdgeLog, rate: float, duration_s: float, seed: int = 5, l_lo: int = 8,
                   l_hi: int = 100):
    """Poisson arrivals at `rate` per second over `duration_s`: a list of
    (arrival_s, Query) with the type uniform over SSSP/SSWP/BFS, a uniform
    source, a window length uniform in [l_lo, l_hi] at a uniform offset."""
    rng = np.random.default_rng(seed)
    l_hi = min(l_hi, log.S)
    t = 0.0
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration_s:
            break
        L = int(rng.integers(l_lo, l_hi + 1))
        b = int(rng.integers(0, log.S - L + 1))
        out.append((t, Query(int(rng.integers(0, 3)), int(rng.integers(0, log.V)), b, L)))
    return out
