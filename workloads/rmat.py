"""Seeded synthetic evolving graphs: an RMAT base graph plus a per-snapshot delta log.

This module only draws random inputs.  It holds none of the stable-vertex-value
method's arithmetic (no bounds, no masks, no relaxation): both the CPU oracle
and the GPU library consume the edge log it returns, each in its own way.

Model (the paper's setting, Section 2): all vertices exist in every snapshot;
snapshot G_0 is the base graph and snapshot G_s (s >= 1) is G_{s-1} after one
batch of edge deletions and one batch of edge additions.  Every added edge is a
new *edge instance* with its own weight; a deleted instance never comes back
(re-adding the same (u, v) pair creates a fresh instance).  Duplicates and
self-loops are kept.

Only ``Generator.integers`` and ``Generator.random`` are used, so a given seed
gives the same log on x86 and on Arm.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


@dataclass
class EdgeLog:
    """An evolving graph as a log of edge instances.

    Instance ``k`` goes from ``src[k]`` to ``dst[k]`` with weight ``w[k]``.
    Step ``s`` (0 <= s < S) first deletes the instances
    ``del_ids[del_off[s]:del_off[s+1]]`` (step 0 deletes nothing) and then adds
    the instances with ids ``add_off[s] .. add_off[s+1]-1`` (step 0 adds the
    base graph).  Snapshot ``G_i`` is the set of instances live after steps
    ``0..i``.  ``t_add[k]``/``t_del[k]`` record the step that added/deleted
    instance ``k`` (``t_del[k] == S`` if it is never deleted), so instance ``k``
    is live in snapshot ``i`` iff ``t_add[k] <= i < t_del[k]``.
    """

    V: int
    S: int
    src: np.ndarray  # uint32 [n_inst]
    dst: np.ndarray  # uint32 [n_inst]
    w: np.ndarray  # uint32 [n_inst]
    add_off: np.ndarray  # int64 [S+1]
    del_off: np.ndarray  # int64 [S+1]
    del_ids: np.ndarray  # int64 [n_del]
    t_add: np.ndarray  # uint32 [n_inst]
    t_del: np.ndarray  # uint32 [n_inst]
    meta: dict = field(default_factory=dict)

    @property
    def n_inst(self) -> int:
        return int(self.src.shape[0])

    @property
    def n_base(self) -> int:
        return int(self.add_off[1])


def rmat_endpoints(rng: np.random.Generator, scale: int, n: int, abcd=RMAT_ABCD):
    """Draw ``n`` RMAT (src, dst) pairs on 2**scale vertices, no noise.

    At every one of the ``scale`` levels (most significant bit first) the
    quadrant is (0,0) with probability a, (0,1) with b, (1,0) with c, (1,1)
    with d; the row bit goes to the source and the column bit to the target.
    """
    a, b, c, _ = abcd
    ab, abc = np.float32(a + b), np.float32(a + b + c)
    fa = np.float32(a)
    src = np.zeros(n, dtype=np.uint32)
    dst = np.zeros(n, dtype=np.uint32)
    for _level in range(scale):
        r = rng.random(n, dtype=np.float32)
        row = r >= ab
        col = ((r >= fa) & ~row) | (r >= abc)
        src <<= np.uint32(1)
        dst <<= np.uint32(1)
        src |= row
        dst |= col
    return src, dst


def _distinct_positions(rng: np.random.Generator, n: int, k: int) -> np.ndarray:
    """``k`` distinct positions in ``[0, n)``, uniformly, in draw order."""
    if k > n:
        raise ValueError(f"cannot delete {k} of {n} live instances")
    taken = np.zeros(n, dtype=bool)
    out = []
    need = k
    while need > 0:
        cand = rng.integers(0, n, size=need + need // 8 + 16, dtype=np.int64)
        # first occurrence of each candidate, in draw order
        _, first = np.unique(cand, return_index=True)
        cand = cand[np.sort(first)]
        cand = cand[~taken[cand]][:need]
        taken[cand] = True
        out.append(cand)
        need -= cand.shape[0]
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int64)


def make_log(
    *,
    scale: int,
    n_edges: int,
    n_snapshots: int,
    n_add: int,
    n_del: int,
    w_lo: int,
    w_hi: int,
    seed: int,
    add_mode: str = "rmat",
    base_mode: str = "rmat",
    abcd=RMAT_ABCD,
) -> EdgeLog:
    """Build an evolving-graph edge log.

    ``w`` is uniform in ``[w_lo, w_hi]`` (inclusive), drawn per instance at
    creation.  The base graph uses ``seed``; step ``s`` draws from
    ``seed * 1000003 + s``.  Deletions are uniform over the live instances.
    ``add_mode`` picks the endpoints of added instances: ``"rmat"`` (RMAT
    draw), ``"uniform"`` (uniform vertices) or ``"skewed"`` (the source of one
    uniformly chosen live instance and the target of another, so additions
    follow the degree distribution).
    """
    V = 1 << scale
    S = int(n_snapshots)
    if S < 1:
        raise ValueError("need at least one snapshot")
    rng0 = np.random.default_rng(seed)
    if base_mode == "rmat":
        bs, bd = rmat_endpoints(rng0, scale, n_edges, abcd)
    elif base_mode == "uniform":
        bs = rng0.integers(0, V, size=n_edges, dtype=np.int64).astype(np.uint32)
        bd = rng0.integers(0, V, size=n_edges, dtype=np.int64).astype(np.uint32)
    else:
        raise ValueError(base_mode)
    bw = rng0.integers(w_lo, w_hi + 1, size=n_edges, dtype=np.int64).astype(np.uint32)

    srcs, dsts, ws = [bs], [bd], [bw]
    t_adds = [np.zeros(n_edges, dtype=np.uint32)]
    add_off = [0, n_edges]
    del_off = [0, 0]
    del_chunks = []
    live = np.arange(n_edges, dtype=np.int64)
    n_total = n_edges
    live_src = bs.copy() if add_mode == "skewed" else None
    live_dst = bd.copy() if add_mode == "skewed" else None
    for s in range(1, S):
        rng = np.random.default_rng(seed * 1000003 + s)
        pos = _distinct_positions(rng, live.shape[0], n_del)
        del_chunks.append(live[pos])
        if add_mode == "rmat":
            as_, ad = rmat_endpoints(rng, scale, n_add, abcd)
        elif add_mode == "uniform":
            as_ = rng.integers(0, V, size=n_add, dtype=np.int64).astype(np.uint32)
            ad = rng.integers(0, V, size=n_add, dtype=np.int64).astype(np.uint32)
        elif add_mode == "skewed":
            p1 = rng.integers(0, live.shape[0], size=n_add, dtype=np.int64)
            p2 = rng.integers(0, live.shape[0], size=n_add, dtype=np.int64)
            as_ = live_src[p1]
            ad = live_dst[p2]
        else:
            raise ValueError(add_mode)
        aw = rng.integers(w_lo, w_hi + 1, size=n_add, dtype=np.int64).astype(np.uint32)
        new_ids = np.arange(n_total, n_total + n_add, dtype=np.int64)
        n_total += n_add
        # deleted positions are refilled by the new instances (order of the
        # live list is arbitrary but deterministic); the surplus is appended
        # or swapped out
        m = min(n_add, n_del)
        live[pos[:m]] = new_ids[:m]
        if add_mode == "skewed":
            live_src[pos[:m]] = as_[:m]
            live_dst[pos[:m]] = ad[:m]
        if n_del > m:
            # the surplus deleted positions take the last live instances
            # (highest position first), so no step copies the whole list
            n_live = live.shape[0]
            for p in np.sort(pos[m:])[::-1].tolist():
                last = n_live - 1
                if p != last:
                    live[p] = live[last]
                    if add_mode == "skewed":
                        live_src[p] = live_src[last]
                        live_dst[p] = live_dst[last]
                n_live -= 1
            live = live[:n_live]
            if add_mode == "skewed":
                live_src = live_src[:n_live]
                live_dst = live_dst[:n_live]
        if n_add > m:
            live = np.concatenate([live, new_ids[m:]])
            if add_mode == "skewed":
                live_src = np.concatenate([live_src, as_[m:]])
                live_dst = np.concatenate([live_dst, ad[m:]])
        srcs.append(as_)
        dsts.append(ad)
        ws.append(aw)
        t_adds.append(np.full(n_add, s, dtype=np.uint32))
        add_off.append(n_total)
        del_off.append(del_off[-1] + n_del)

    del_ids = np.concatenate(del_chunks) if del_chunks else np.zeros(0, dtype=np.int64)
    t_del = np.full(n_total, S, dtype=np.uint32)
    for s in range(1, S):
        t_del[del_ids[del_off[s]:del_off[s + 1]]] = s
    return EdgeLog(
        V=V,
        S=S,
        src=np.concatenate(srcs).astype(np.uint32),
        dst=np.concatenate(dsts).astype(np.uint32),
        w=np.concatenate(ws).astype(np.uint32),
        add_off=np.asarray(add_off, dtype=np.int64),
        del_off=np.asarray(del_off, dtype=np.int64),
        del_ids=del_ids.astype(np.int64),
        t_add=np.concatenate(t_adds).astype(np.uint32),
        t_del=t_del,
        meta=dict(scale=scale, n_edges=n_edges, n_add=n_add, n_del=n_del, w_lo=w_lo,
                  w_hi=w_hi, seed=seed, add_mode=add_mode, base_mode=base_mode),
    )


def max_out_degree_vertex(log: EdgeLog) -> int:
    """Vertex with the most live out-edge instances in G_0 (smallest id on ties)."""
    deg = np.bincount(log.src[: log.n_base].astype(np.int64), minlength=log.V)
    return int(np.argmax(deg))


def random_small_log(seed: int, V: int, n_edges: int, S: int, n_add: int, n_del: int,
                     w_lo: int = 1, w_hi: int = 20) -> EdgeLog:
    """Tiny uniform evolving graph for brute-force checks (V need not be a power of 2)."""
    rng0 = np.random.default_rng(seed)
    bs = rng0.integers(0, V, size=n_edges, dtype=np.int64).astype(np.uint32)
    bd = rng0.integers(0, V, size=n_edges, dtype=np.int64).astype(np.uint32)
    bw = rng0.integers(w_lo, w_hi + 1, size=n_edges, dtype=np.int64).astype(np.uint32)
    srcs, dsts, ws, t_adds = [bs], [bd], [bw], [np.zeros(n_edges, np.uint32)]
    add_off, del_off, dels = [0, n_edges], [0, 0], []
    live = np.arange(n_edges, dtype=np.int64)
    n_total = n_edges
    for s in range(1, S):
        rng = np.random.default_rng(seed * 1000003 + s)
        k = min(n_del, live.shape[0])
        pos = _distinct_positions(rng, live.shape[0], k)
        dels.append(live[pos])
        keep = np.ones(live.shape[0], dtype=bool)
        keep[pos] = False
        as_ = rng.integers(0, V, size=n_add, dtype=np.int64).astype(np.uint32)
        ad = rng.integers(0, V, size=n_add, dtype=np.int64).astype(np.uint32)
        aw = rng.integers(w_lo, w_hi + 1, size=n_add, dtype=np.int64).astype(np.uint32)
        live = np.concatenate([live[keep], np.arange(n_total, n_total + n_add)])
        n_total += n_add
        srcs.append(as_)
        dsts.append(ad)
        ws.append(aw)
        t_adds.append(np.full(n_add, s, np.uint32))
        add_off.append(n_total)
        del_off.append(del_off[-1] + k)
    del_ids = np.concatenate(dels) if dels else np.zeros(0, np.int64)
    t_del = np.full(n_total, S, dtype=np.uint32)
    for s in range(1, S):
        t_del[del_ids[del_off[s]:del_off[s + 1]]] = s
    return EdgeLog(V=V, S=S, src=np.concatenate(srcs).astype(np.uint32),
                   dst=np.concatenate(dsts).astype(np.uint32),
                   w=np.concatenate(ws).astype(np.uint32),
                   add_off=np.asarray(add_off, np.int64), del_off=np.asarray(del_off, np.int64),
                   del_ids=del_ids.astype(np.int64), t_add=np.concatenate(t_adds),
                   t_del=t_del, meta=dict(seed=seed, V=V, kind="small-uniform"))
