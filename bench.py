#!/usr/bin/env python
"""Benchmark: snapshot x vertex values per second of the intersection-union
path on one GB300, against the plain per-snapshot GPU recompute and the CPU
oracle.

Workload (default ``rmat20``): RMAT scale 20 (1,048,576 vertices, 16,777,216
edges, a/b/c = 0.57/0.19/0.19), weights uniform in [1, 999], 64 snapshots, each
step deleting 10,000 uniform live edges and adding 10,000 RMAT edges.  One
step = an SSSP query and an SSWP query from the highest-out-degree vertex of
G_0 over the window [0, 64), each through the whole path (intersection solve,
union solve, stable compaction + subgraph extraction, multi-snapshot
relaxation, scatter to a 64 x V uint32 device array).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import gc as pygc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "snapshot x vertex values/s (intersection-union query path)"
UNIT = "values/s"
L2_BYTES = 129 * 1024 * 1024


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["svv", "reference"], default="svv")
    p.add_argument("--workload", choices=["rmat20", "small", "batch22", "batch20", "batch16", "rmat24", "serve22",
                                          "serve16", "sensitivity", "ablation"],
                   default="rmat20",
                   help="rmat20: the headline line; batch*: many mixed queries in one launch; rmat24: the "
                        "two-mask-word scale-24 graph; serve*: Poisson request streams")
    p.add_argument("--serve-seconds", type=float, default=10.0)
    p.add_argument("--plain-steps", type=int, default=1, help="timed steps of the plain recompute (0 = skip)")
    p.add_argument("--step-api", choices=["groups", "async"], default="groups",
                   help="rmat20/small: the step's queries in one svv_query_batch call as one query group of "
                        "mixed types (groups), or one svv_query_async call per query (async)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--tune", action="append", default=[], metavar="KEY=VALUE",
                   help="library tuning knob (svv_set_tuning), repeatable")
    p.add_argument("--batch-queries", type=int, default=0,
                   help="batch*: number of queries (default: the workload's own)")
    p.add_argument("--batch-max-len", type=int, default=0,
                   help="batch*: cap every window at this many snapshots (a small case of the same mix)")
    p.add_argument("--autotune", action="store_true",
                   help="batch*/serve*: run svv_autotune per query type and window-length bucket before warm-up")
    p.add_argument("--verbose", action="store_true")
    return p.parse_args()


def make_workload(name):
    if name == "small":
        log = W.small_rmat()
        qs = [W.Query(W.SSSP, 0, 0, log.S), W.Query(W.SSWP, 0, 0, log.S)]
        desc = "RMAT V=4096 E=32768 w[1,255] S=8, 1% churn/step; SSSP+SSWP from 0, window [0,8)"
    else:
        log = W.rmat20()
        qs = W.rmat20_queries(log)
        desc = ("RMAT scale 20 (V=1,048,576, E0=16,777,216) w[1,999] S=64, 10k del + 10k RMAT add per step; "
                "SSSP+SSWP from the max-out-degree vertex, window [0,64)")
    return log, qs, desc


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [x for x in sm if mx and x > 0.3 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def gpu_id_of(dev):
    import torch
    try:
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


# ---------------------------------------------------------------------------
def graph_counts(log, rp, mask):
    S = log.S
    Wd = (S + 63) // 64
    m = mask.reshape(-1, Wd)
    full = np.ones(m.shape[0], bool)
    for j in range(Wd):
        n = min(64, S - 64 * j)
        hist = np.uint64((1 << n) - 1) if n < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        full &= (m[:, j] & hist) == hist
    return {"V": log.V, "E": int(m.shape[0]), "NF": int((~full).sum()), "W": Wd}


def algorithmic_bytes(phase, gc, st, L):
    """Algorithmic bytes of one launch of a phase by the per-unit figures of
    the hot-path table (instances of 8 + 8W bytes, values and row offsets):
    each bound solve makes one pass over the union graph, the compaction reads
    both bounds and filters the graph, the relaxation reads the subgraph once
    and reads and updates every row, the scatter writes the L x V result."""
    V, E, Wd = gc["V"], gc["E"], gc["W"]
    U, EQ = (st["unstable"], st["qrs_edges"]) if st else (0, 0)
    QW = (L + 63) // 64
    if phase in ("cap", "cup"):
        return 8 * V + E * (8 + 8 * Wd) + 4 * V
    if phase == "qrs":
        return 8 * V + V / 8 + E * (4 + 8 * Wd) + EQ * (8 + 8 * QW)
    if phase == "relax":
        return EQ * (8 + 8 * QW) + 2 * U * L * 4
    if phase == "scatter":
        return L * V * 4
    if phase == "plain":
        return L * (8 * V + E * (8 + 8 * Wd) + 4 * V) + L * V * 4
    return 0


def layout_bytes(phase, gc, st, L):
    """The floor of the resident layout (8 B per edge, 8 B per mask word of an
    edge not present in every snapshot, 8 B of row offsets and 4 B of value
    per vertex): what each kernel must move at least with this layout."""
    V, E, NF, Wd = gc["V"], gc["E"], gc["NF"], gc["W"]
    U, EQ, EM = st["unstable"], st["qrs_edges"], st["qrs_masked"]
    QW = (L + 63) // 64
    LP = 8 if L <= 8 else 16 if L <= 16 else 32 if L <= 32 else 64 if L <= 64 else 128
    if phase == "cap":  # one pass over the edges present in every snapshot
        return 8 * (V + 1) + 8 * (E - NF) + 4 * V
    if phase == "cup":  # addition edges, then one pass over the union graph
        return NF * (4 + 8 + 8 * Wd) + 8 * (V + 1) + 8 * E + 8 * NF * Wd + 8 * V
    if phase == "qrs":  # compare bounds, read unstable rows twice, write the subgraph
        return 8 * V + 8 * V + 2 * (8 * EQ) + 8 * EQ + 8 * QW * EM + 16 * U
    if phase == "relax":  # init rows, seed list, one pass over the subgraph edges and rows
        return 4 * U * LP + NF * (4 + 8 + 8 * Wd) + 8 * EQ + 8 * QW * EM + 2 * 4 * U * LP
    if phase == "scatter":
        return 4 * L * V + 8 * V + 4 * U * LP
    return 0


def group_layout_bytes(phase, gc, n):
    """The floor of one group solve of n queries: the graph once, n values
    per vertex."""
    V, E, NF, Wd = gc["V"], gc["E"], gc["NF"], gc["W"]
    if phase == "cap":
        return 8 * (V + 1) + 8 * (E - NF) + 4 * n * V
    if phase == "cup":
        return NF * (4 + 8 + 8 * Wd) + 8 * (V + 1) + 8 * E + 8 * NF * Wd + 8 * n * V
    return 0


PHASE_KERNELS = {"cap": "solve_kernel<Op, kPredAll> (intersection graph)",
                 "cup": "solve_kernel<Op, kPredAny> (union graph)",
                 "qrs": "qrs_kernel (stable compaction + subgraph)",
                 "relax": "relax_kernel<Op, P, K> (Algorithm 2)",
                 "scatter": "scatter_kernel (output)"}


GROUP_KERNELS = {"cap": "group_solve_kernel<OpMixed, KL, kPredAll> (intersection graphs of the step's queries, "
                        "one launch)",
                 "cup": "group_solve_kernel<OpMixed, KL, kPredAny> (union graphs of the step's queries, one launch)"}

# kernel -> (profile summary holding its traffic line, sources whose hash it names)
KERNEL_SOURCES = {"cap": ("solve_kernel_rmat20.md",
                          ["svv_solve.cu", "svv_solve.cuh", "svv_team.cuh", "svv_device.cuh", "svv_push.cuh",
                           "svv_internal.h"]),
                  "group_cap": ("group_solve_kernel_rmat20_pair.md",
                                ["svv_group.cu", "svv_group.cuh", "svv_team.cuh", "svv_device.cuh", "svv_push.cuh",
                                 "svv_internal.h"])}


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, only while the
    kernel's sources still hash to the version that was captured."""
    import hashlib
    import re
    if workload != "rmat20" or kernel not in KERNEL_SOURCES:
        return None
    prof, srcs = KERNEL_SOURCES[kernel]
    h = hashlib.sha256()
    for f in srcs:
        with open(os.path.join(ROOT, "paper_2502_10579_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    try:
        with open(os.path.join(ROOT, "profiles", prof)) as fh:
            for line in fh:
                m = re.match(r"traffic: kernel=(\w+) bytes_per_launch=(\d+) sources_sha256=(\w+)", line.strip())
                if m and m.group(1) == kernel and m.group(3) == h.hexdigest():
                    return int(m.group(2))
    except OSError:
        pass
    return None


def _isolated(log, source):
    """True when the source has no out-edge in any snapshot."""
    deg = getattr(log, "_outdeg", None)
    if deg is None:
        deg = np.bincount(np.asarray(log.src, np.int64), minlength=log.V)
        log._outdeg = deg
    return bool(deg[source] == 0)


def _len_bucket(L):
    """Window-length bucket of the library's tuned knobs (up to 8, 16, 32, 64, more)."""
    return 0 if L <= 8 else 1 if L <= 16 else 2 if L <= 32 else 3 if L <= 64 else 4


def _autotune(svv, ctx, log, qs):
    """svv_autotune on one probe query (the first with a source that has
    out-edges) of every (type, window-length bucket) in qs; returns the knobs
    it kept, keyed by type and bucket bound."""
    probes = {}
    for q in qs:
        key = (q.type, _len_bucket(q.win_len))
        if key not in probes and not _isolated(log, q.source):
            probes[key] = q
    bound = ["<=8", "<=16", "<=32", "<=64", ">64"]
    out = {}
    for (t, b), q in sorted(probes.items()):
        r = svv.svv_autotune(ctx.h, t, q.source, q.win_begin, q.win_len, reps=2)
        out[f"{W.TYPE_NAMES[t]}_L{bound[b]}"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()}
    return out


def _batch_launches(log, qs, gmax):
    """Kernel launches of an in-order batch: a query whose source has no
    out-edge is one fill; the others run in groups of up to gmax of one type
    (lane words, two group solves, split) and then three kernels each
    (compaction + extraction, relaxation, scatter; a group of one runs the
    five kernels of a single query)."""
    n, open_ = 0, {}
    groups = []
    for q in qs:
        if _isolated(log, q.source):
            n += 1
            continue
        g = open_.get(q.type)
        if g is None or len(g) >= gmax:
            g = []
            open_[q.type] = g
            groups.append(g)
        g.append(q)
    for g in groups:
        n += 5 if len(g) == 1 else 4 + 3 * len(g)
    return n


def cpu_baseline(log, qs, nthreads=0, snaps=None, single_core=True):
    """The oracle on the host cores (threads over snapshots), and on one core."""
    import oracle
    cores = nthreads or os.cpu_count() or 1
    k = snaps or max(2, min(log.S, cores // len(qs) if cores >= len(qs) else 1))
    t0 = time.perf_counter()
    vals = 0
    for q in qs:
        oracle.query(log, q.type, q.source, q.win_begin, k, nthreads=cores)
        vals += k * log.V
    dt = time.perf_counter() - t0
    out = {"value": vals / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{len(qs)} queries x {k} snapshots (of {qs[0].win_len}) from scratch, "
                     f"threads over snapshots, {dt:.2f} s wall"}
    if single_core:
        t0 = time.perf_counter()
        for q in qs:
            oracle.query(log, q.type, q.source, q.win_begin, 1, nthreads=1)
        dt1 = time.perf_counter() - t0
        out["single_core"] = {"value": len(qs) * log.V / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"{len(qs)} queries x 1 snapshot on one core, {dt1:.2f} s"}
    return out


# ---------------------------------------------------------------------------
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, world, rank):
    log, qs, desc = make_workload(args.workload)
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    k = max(1, min(log.S, cores // 2))
    for _ in range(args.warmup):
        pass  # the oracle has no warm state: warm-up steps are not repeated
    times, vals = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(log, qs, cores, k, single_core=False)
        times.append(time.perf_counter() - t0)
        vals += len(qs) * k * log.V
    total = sum(times)
    value = vals / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": desc, "sample_snapshots": k},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": cb["sample"],
                             "single_core": cpu_baseline(log, qs, 1, 1)["single_core"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _setup_ctx(svv, log, dev, args):
    rp, col, w, mask = svv.svv_build_versioned_csr(log.V, log.S, log.src, log.dst, log.w, log.t_add, log.t_del)
    ctx = svv.Context(dev)
    _tune(ctx, args)
    ctx.load_csr(log.V, log.S, rp, col, w, mask)
    return ctx


def _tune(ctx, args):
    """--tune knobs, set before the graph is loaded (chunk sizes and the
    transposed graph are fixed at load)."""
    for kv in args.tune:
        k, v = kv.split("=", 1)
        ctx.set_tuning(k, int(v))


def _tuning(args, tuned=None):
    """config.tuning: the --tune knobs, and what the autotuner kept."""
    d = dict(kv.split("=", 1) for kv in args.tune)
    if tuned is not None:
        d["autotuned"] = tuned
    return d


def _clocks_start(rank, args, dev):
    s = ClockSampler(gpu_id_of(dev)) if (rank == 0 and not args.no_clocks) else None
    if s:
        s.start()
    return s


def run_batch(args, world, rank, local):
    """Many mixed queries (1/3 each type, uniform sources, window lengths
    uniform in [8, 64] at uniform offsets) answered by ONE svv_query_batch
    launch; one step = the whole batch."""
    import torch

    import __graft_entry__
    from paper_2502_10579_gb300 import svv
    dev = local
    torch.cuda.set_device(dev)
    __graft_entry__.build()
    if args.workload == "batch22":
        log, nq = W.rmat22(), 256
        desc = "RMAT scale 22 (V=4,194,304, E0=67,108,864) w[1,999] S=64, 0.05% churn/step; 256 mixed queries, L in [8,64]"
    elif args.workload == "batch20":
        log, nq = W.rmat20(), 16
        desc = ("RMAT scale 20 (V=1,048,576, E0=16,777,216) w[1,999] S=64, 10k del + 10k RMAT add per step; "
                "16 mixed queries, L in [8,64]")
        args.tune = ["batch_mode=2"] + list(args.tune)  # query groups at this size too
    else:
        log, nq = W.scaled_rmat(16, 16, 64, 0.0005, 1016), 64
        desc = "RMAT scale 16 (V=65,536, E0=1,048,576) w[1,999] S=64, 0.05% churn/step; 64 mixed queries, L in [8,64]"
    if args.batch_queries:
        nq = args.batch_queries
        desc += f"; this run: {nq} queries of the same mix"
    qs = W.batch_queries(log, n=nq, seed=3)
    if args.batch_max_len:
        qs = [W.Query(q.type, q.source, q.win_begin, min(q.win_len, args.batch_max_len)) for q in qs]
        desc += f"; windows capped at {args.batch_max_len} snapshots"
    ctx = _setup_ctx(svv, log, dev, args)
    tuned = _autotune(svv, ctx, log, qs) if args.autotune else None
    outs = [ctx.empty_out(q.win_len) for q in qs]
    specs = [(q.type, q.source, q.win_begin, q.win_len, o) for q, o in zip(qs, outs)]
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(1, args.warmup)):
        st = svv.svv_query_batch(ctx.h, specs, stream)
        assert all(x == 0 for x in st), st
    torch.cuda.synchronize()
    sampler = _clocks_start(rank, args, dev)
    barrier(world)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for _ in range(args.steps):
        ev0.record(stream)
        svv.svv_query_batch(ctx.h, specs, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms += ev0.elapsed_time(ev1)
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(ms, world, f"cuda:{dev}")
    vals = sum(q.win_len * log.V for q in qs)
    value = vals * args.steps * world / (ms / 1e3)
    stats = ctx.stats()
    one_launch = stats["batch_teams"] > 0
    # the same queries one at a time through svv_query, and a sample of the
    # plain per-snapshot recompute
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for q, o in zip(qs, outs):
        ctx.query(q.type, q.source, q.win_begin, q.win_len, out=o, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    sample = qs[:6]
    e0.record(stream)
    for q in sample:
        ctx.query(q.type, q.source, q.win_begin, q.win_len, stream=stream, plain=True)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    plain_value = sum(q.win_len * log.V for q in sample) / (plain_ms / 1e3)
    if rank == 0:
        print(json.dumps({
            "metric": "snapshot x vertex values/s (batched intersection-union queries, svv_query_batch)",
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": desc, "queries": nq, "output_bytes": int(vals * 4),
                       "mode": "one launch" if one_launch else "in order",
                       "teams": stats["batch_teams"], "team_blocks": stats["batch_team_blocks"],
                       "tuning": _tuning(args, tuned)},
            "one_at_a_time": {"value": vals / (seq_ms / 1e3), "unit": UNIT, "ms": seq_ms},
            "plain_sample": {"value": plain_value, "unit": UNIT, "queries": len(sample), "ms": plain_ms},
            "clocks": clocks,
            "gpu_launches": args.steps * (1 if one_launch else _batch_launches(log, qs, 8))}), flush=True)
    ctx.close()
    return 0


def run_rmat24(args, world, rank, local):
    """RMAT scale 24, 100 snapshots (two mask words), SSSP and BFS from 16
    sources at windows of 25, 50 and 100 snapshots, one query at a time."""
    import torch

    import __graft_entry__
    from paper_2502_10579_gb300 import svv
    dev = local
    torch.cuda.set_device(dev)
    __graft_entry__.build()
    t0 = time.perf_counter()
    log = W.rmat24()
    gen_s = time.perf_counter() - t0
    qs = W.rmat24_queries(log)
    ctx = _setup_ctx(svv, log, dev, args)
    ctx.set_tuning("phase_timing", 1)
    out = ctx.empty_out(max(q.win_len for q in qs))
    stream = torch.cuda.current_stream(dev)
    for q in qs[:2]:
        ctx.query(q.type, q.source, q.win_begin, q.win_len, out=out[: q.win_len], stream=stream)
    torch.cuda.synchronize()
    sampler = _clocks_start(rank, args, dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per = []
    for q in qs:
        e0.record(stream)
        ctx.query(q.type, q.source, q.win_begin, q.win_len, out=out[: q.win_len], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        st = ctx.stats()
        per.append((q.type, q.win_len, e0.elapsed_time(e1), st["unstable"], st["qrs_edges"]))
    clocks = sampler.stop() if sampler else None
    ms = sum(p[2] for p in per)
    vals = sum(q.win_len * log.V for q in qs)
    by = {}
    for t, L, m, u, eq in per:
        k = f"{W.TYPE_NAMES[t]}_L{L}"
        by.setdefault(k, []).append(m)
    if rank == 0:
        print(json.dumps({
            "metric": "snapshot x vertex values/s (intersection-union path, scale-24 graph)",
            "value": vals * world / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": len(qs), "warmup": 2,
            "ms_per_step": ms / len(qs), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": "RMAT scale 24 (V=16,777,216, E0=268,435,456) w[1,999] S=100 (2 mask words), "
                                   "0.1% degree-skewed churn/step; SSSP+BFS x 16 sources x L in {25,50,100}",
                       "generate_s": gen_s, "edges": ctx.graph.E},
            "ms_by_query_kind": {k: statistics.median(v) for k, v in by.items()},
            "clocks": clocks, "gpu_launches": 5 * len(qs)}), flush=True)
    ctx.close()
    return 0


def run_serve(args, world, rank, local):
    """Poisson request streams at 100, 1,000 and 10,000 requests/s (type
    uniform, source uniform, L uniform in [8, 100] at a uniform offset) served
    with arena admission -- by the live batch kernel below 2M vertices, in
    query groups from 2M (up to 8 same-type requests share the bound solves,
    then each runs its own extraction, relaxation and scatter); the plain
    per-snapshot recompute served FIFO on the first requests of the 100/s
    stream."""
    import torch

    import __graft_entry__
    from paper_2502_10579_gb300 import svv
    dev = local
    torch.cuda.set_device(dev)
    __graft_entry__.build()
    if args.workload == "serve22":
        log = W.rmat22(seed=1005, n_snapshots=128)
        desc = "RMAT scale 22 (V=4,194,304, E0=67,108,864) w[1,999] S=128, 0.05% churn/step"
    else:
        log = W.scaled_rmat(16, 16, 128, 0.0005, 1016)
        desc = "RMAT scale 16 (V=65,536, E0=1,048,576) w[1,999] S=128, 0.05% churn/step"
    ctx = _setup_ctx(svv, log, dev, args)
    tuned = _autotune(svv, ctx, log, [q for _, q in W.serve_requests(log, 1000, 1.0, seed=5)]) if args.autotune else None
    arena = (64 << 30) if args.workload == "serve22" else (2 << 30)
    svv.svv_serve_start(ctx.h, max_window=min(100, log.S), capacity=1 << 16, arena_bytes=arena)
    bm = int(dict(kv.split("=", 1) for kv in args.tune).get("batch_mode", 0))
    gm = int(dict(kv.split("=", 1) for kv in args.tune).get("group_max", 8))
    mode = (("query groups of up to %d" % gm if gm > 1 else "in order")
            if bm == 2 or (bm == 0 and log.V >= (2 << 20)) else "live kernel")
    dur = args.serve_seconds
    warm = 1.0
    results = {}
    for rate in (100, 1000, 10000):
        # a saturated stream only grows its backlog: cap each stream at about
        # 2,500 requests; the first 10% are warm-up and not measured
        d = min(dur + warm, 2500.0 / rate)
        reqs = W.serve_requests(log, rate, d, seed=5)
        warm = 0.1 * d
        lat, done = svv.svv_serve_replay(ctx.h, [(a, q.type, q.source, q.win_begin, q.win_len) for a, q in reqs])
        arr = np.array([a for a, _ in reqs])
        meas = arr >= warm
        span = (done[meas].max() - warm) if meas.any() else 1.0
        vals = sum(q.win_len * log.V for (a, q), m in zip(reqs, meas) if m)
        results[str(rate)] = {"requests": int(meas.sum()), "p50_ms": float(np.percentile(lat[meas], 50)),
                              "p99_ms": float(np.percentile(lat[meas], 99)),
                              "throughput_rps": float(meas.sum() / span), "values_per_s": vals / span}
    svv.svv_serve_stop(ctx.h)
    # plain per-snapshot recompute served FIFO, first requests of the 100/s stream
    reqs = W.serve_requests(log, 100, 1.0, seed=5)[:12]
    out = ctx.empty_out(min(100, log.S))
    t_start = time.perf_counter()
    lat = []
    for arr, q in reqs:
        while time.perf_counter() - t_start < arr:
            time.sleep(0.0001)
        ctx.query(q.type, q.source, q.win_begin, q.win_len, out=out[: q.win_len], plain=True)
        torch.cuda.synchronize()
        lat.append(1e3 * (time.perf_counter() - t_start - arr))
    span = time.perf_counter() - t_start - reqs[0][0]
    plain = {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
             "throughput_rps": len(reqs) / span,
             "values_per_s": sum(q.win_len * log.V for _, q in reqs) / span}
    if rank == 0:
        best = max(results.values(), key=lambda r: r["values_per_s"])
        print(json.dumps({
            "metric": "served requests: p50/p99 latency ms and throughput under Poisson arrivals",
            "value": best["values_per_s"], "unit": UNIT, "n_gpus": world, "steps": sum(r["requests"] for r in results.values()),
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": desc + f"; Poisson 100/1,000/10,000 req/s, each stream min({dur:g} s, 2,500 requests), "
                                   "first 10% excluded",
                       "arena_bytes": arena, "admission": "output arena (svv_submit refuses when full)",
                       "mode": mode, "tuning": _tuning(args, tuned)},
            "serve": results, "plain_fifo": plain}), flush=True)
    ctx.close()
    return 0


def run_ablation(args, world, rank, local):
    """The execution modes of the paper's Table 3 on the scale-20 workload,
    SSSP and SSWP over the whole history, on one GB300: the intersection-union
    path with all snapshots relaxed together (CQRS), the same subgraph relaxed
    one snapshot per pass (QRS: slab_max = 1), direct-hop evaluation from the
    intersection values without stable-vertex pruning (CG: prune = 0), and
    the plain per-snapshot recompute.  Every mode gives identical values."""
    import torch

    import __graft_entry__
    from paper_2502_10579_gb300 import svv
    dev = local
    torch.cuda.set_device(dev)
    __graft_entry__.build()
    log = W.rmat20()
    qs = W.rmat20_queries(log)
    ctx = _setup_ctx(svv, log, dev, args)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=f"cuda:{dev}")
    outs = [ctx.empty_out(q.win_len) for q in qs]
    modes = [("CQRS", "intersection-union, all window snapshots relaxed together", {}, False),
             ("QRS", "same subgraph, one snapshot per relaxation pass (slab_max=1)", {"slab_max": 1}, False),
             ("CG", "direct-hop from the intersection values, no stable-vertex pruning (prune=0)", {"prune": 0},
              False),
             ("plain", "full solve of every snapshot", {}, True)]
    table = []
    for name, what, knobs, plain in modes:
        for k, v in knobs.items():
            ctx.set_tuning(k, v)
        per = {}
        for q, o in zip(qs, outs):
            steps = 1 if plain else max(1, args.steps)
            ctx.query(q.type, q.source, q.win_begin, q.win_len, out=o, stream=stream, plain=plain)  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms = 0.0
            for _ in range(steps):
                flush.zero_()
                e0.record(stream)
                ctx.query(q.type, q.source, q.win_begin, q.win_len, out=o, stream=stream, plain=plain)
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
            per[W.TYPE_NAMES[q.type]] = ms / steps
        for k in knobs:
            ctx.set_tuning(k, {"slab_max": 128, "prune": 1}[k])
        table.append({"mode": name, "what": what, "ms_per_query": per})
    base = {k: v for k, v in table[0]["ms_per_query"].items()}
    for row in table:
        row["cqrs_speedup"] = {k: row["ms_per_query"][k] / base[k] for k in base}
    vals = sum(q.win_len * log.V for q in qs)
    best = vals / (sum(base.values()) / 1e3)
    if rank == 0:
        print(json.dumps({
            "metric": "ms per query by execution mode (the paper's Table 3 rows on one GB300)", "value": best,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": 1, "ms_per_step": sum(base.values()),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "RMAT scale 20 (V=1,048,576, E0=16,777,216) w[1,999] S=64, 10k del + 10k RMAT "
                                   "add per step; SSSP+SSWP from the max-out-degree vertex, window [0,64)",
                       "l2": "flushed before every timed query"},
            "table": table}), flush=True)
    ctx.close()
    return 0


def run_sensitivity(args, world, rank, local):
    """How the path responds to the number of snapshots and to the churn per
    step (the paper's sensitivity study, Section 6): RMAT scale 20, S in {32,
    64, 128} x {2,500, 10,000, 40,000} deletions + as many RMAT additions per
    step; SSSP+SSWP from the max-out-degree vertex over the whole history, IU
    against the plain per-snapshot recompute, with the unstable share."""
    import torch

    import __graft_entry__
    from paper_2502_10579_gb300 import svv
    dev = local
    torch.cuda.set_device(dev)
    __graft_entry__.build()
    stream = torch.cuda.current_stream(dev)
    table = []
    for S in (32, 64, 128):
        for churn in (2500, 10000, 40000):
            log = W.make_log(scale=20, n_edges=1 << 24, n_snapshots=S, n_add=churn, n_del=churn, w_lo=1,
                             w_hi=999, seed=1002, add_mode="rmat")
            qs = W.rmat20_queries(log)
            ctx = _setup_ctx(svv, log, dev, args)
            outs = [ctx.empty_out(q.win_len) for q in qs]

            def step(plain=False):
                for q, o in zip(qs, outs):
                    ctx.query(q.type, q.source, q.win_begin, q.win_len, out=o, stream=stream, plain=plain)

            for _ in range(max(1, args.warmup)):
                step()
            unstable = []
            for q, o in zip(qs, outs):
                ctx.query(q.type, q.source, q.win_begin, q.win_len, out=o, stream=stream)
                unstable.append(ctx.stats()["unstable"] / log.V)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            e0.record(stream)
            step(plain=True)
            e1.record(stream)
            torch.cuda.synchronize()
            pms = e0.elapsed_time(e1)
            vals = sum(q.win_len * log.V for q in qs)
            table.append({"snapshots": S, "churn_per_step": 2 * churn, "ms_per_step": ms,
                          "values_per_s": vals / (ms / 1e3), "plain_values_per_s": vals / (pms / 1e3),
                          "iu_speedup": pms / ms, "unstable_share": unstable})
            ctx.close()
            del outs
    if rank == 0:
        best = max(r["values_per_s"] for r in table)
        print(json.dumps({
            "metric": "snapshot x vertex values/s vs snapshots and churn (sensitivity)", "value": best,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "RMAT scale 20 (V=1,048,576, E0=16,777,216) w[1,999], S in {32,64,128} x "
                                   "churn in {5k, 20k, 80k} edge changes per step; SSSP+SSWP, whole history"},
            "table": table}), flush=True)
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload in ("batch22", "batch20", "batch16"):
        return run_batch(args, world, rank, local)
    if args.workload == "rmat24":
        return run_rmat24(args, world, rank, local)
    if args.workload in ("serve22", "serve16"):
        return run_serve(args, world, rank, local)
    if args.workload == "sensitivity":
        return run_sensitivity(args, world, rank, local)
    if args.workload == "ablation":
        return run_ablation(args, world, rank, local)

    import torch

    import __graft_entry__
    from paper_2502_10579_gb300 import svv

    dev = local
    torch.cuda.set_device(dev)
    if rank == 0:
        __graft_entry__.build()
    barrier(world)
    if rank != 0:
        __graft_entry__.build()  # no-op when rank 0 already built

    log, qs, desc = make_workload(args.workload)
    rp, col, w, mask = svv.svv_build_versioned_csr(log.V, log.S, log.src, log.dst, log.w, log.t_add, log.t_del)
    gc = graph_counts(log, rp, mask)
    ctx = svv.Context(dev)
    _tune(ctx, args)
    ctx.load_csr(log.V, log.S, rp, col, w, mask)
    outs = [ctx.empty_out(q.win_len) for q in qs]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)
    groups = args.step_api == "groups"
    if groups:  # the step's queries share one query group whatever their types
        ctx.set_tuning("batch_mode", 2)
        ctx.set_tuning("group_mix", 1)
    specs = [(q.type, q.source, q.win_begin, q.win_len, o) for q, o in zip(qs, outs)]

    def step_groups():
        """One step: the step's queries in one svv_query_batch call (one query
        group of mixed types), which returns after the step."""
        st = svv.svv_query_batch(ctx.h, specs, stream)
        if any(st):
            raise RuntimeError(f"batched step failed: {st}")

    def step_async():
        """One step: every query queued on the stream (svv_query_async), no host wait."""
        return [svv.svv_query_async(ctx.h, q.type, q.source, q.win_begin, q.win_len, o, stream)
                for q, o in zip(qs, outs)]

    def step(plain=False):
        sts = []
        for q, o in zip(qs, outs):
            ctx.query(q.type, q.source, q.win_begin, q.win_len, out=o, stream=stream, plain=plain)
            sts.append(ctx.stats())
        return sts

    for _ in range(args.warmup):
        if groups:
            step_groups()
        else:
            for tk in step_async():
                svv.svv_query_wait(ctx.h, tk)
        flush.zero_()
    torch.cuda.synchronize()

    sampler = ClockSampler(gpu_id_of(dev)) if (rank == 0 and not args.no_clocks) else None
    if sampler:
        sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    tickets = []
    pygc.disable()  # keep collector pauses out of the timed steps
    for i in range(args.steps):
        starts[i].record(stream)
        if groups:
            step_groups()
        else:
            tickets += step_async()
        ends[i].record(stream)
        flush.zero_()  # L2 flush between timed steps, outside the event pair
        if len(tickets) > 32:  # the library keeps 64 queries in flight
            for tk in tickets[:-16]:
                svv.svv_query_wait(ctx.h, tk)
            tickets = tickets[-16:]
    torch.cuda.synchronize()
    pygc.enable()
    for tk in tickets:
        svv.svv_query_wait(ctx.h, tk)  # raises if a query failed
    barrier(world)
    clocks = sampler.stop() if sampler else None
    ms_total = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms_total = max_over_ranks(ms_total, world, f"cuda:{dev}")
    values_per_step = sum(q.win_len * log.V for q in qs)
    value = values_per_step * args.steps * world / (ms_total / 1e3)

    # per-phase device times (CUDA events between the phases on the query
    # stream) in separate, untimed steps of the same queries
    ctx.set_tuning("phase_timing", 1)
    phase_ms = {k: 0.0 for k in ("cap", "cup", "qrs", "relax", "scatter")}
    all_stats = []
    nphase = max(3, min(args.steps, 10))
    for _ in range(nphase):
        sts = step()
        flush.zero_()
        for st in sts:
            for k in phase_ms:
                phase_ms[k] += st["ms_" + k]
        all_stats.append(sts)
    torch.cuda.synchronize()
    # the group solves of the batched step, timed by the library
    group_ms = {"cap": 0.0, "cup": 0.0}
    if groups:
        for _ in range(nphase):
            step_groups()
            gst = ctx.stats()
            group_ms["cap"] += gst["ms_group_cap"]
            group_ms["cup"] += gst["ms_group_cup"]
            flush.zero_()
        torch.cuda.synchronize()
    ctx.set_tuning("phase_timing", 0)

    # plain per-snapshot recompute on the same queries
    plain = None
    if args.plain_steps > 0:
        step(plain=True)
        torch.cuda.synchronize()
        barrier(world)
        ps = torch.cuda.Event(enable_timing=True)
        pe = torch.cuda.Event(enable_timing=True)
        pms = 0.0
        for _ in range(args.plain_steps):
            flush.zero_()
            ps.record(stream)
            step(plain=True)
            pe.record(stream)
            torch.cuda.synchronize()
            pms += ps.elapsed_time(pe)
        pms = max_over_ranks(pms, world, f"cuda:{dev}")
        pvalue = values_per_step * args.plain_steps * world / (pms / 1e3)
        pbytes = sum(algorithmic_bytes("plain", gc, None, q.win_len) for q in qs)
        plain = {"value": pvalue, "unit": UNIT, "ms_per_step": pms / args.plain_steps,
                 "iu_speedup": value / pvalue, "algorithmic_gbs": pbytes / (pms / args.plain_steps / 1e3) / 1e9}

    # end to end through the public API with host output buffers: the step's
    # queries in one svv_query_batch call (each result copied back while the
    # next query computes); the same through svv_query_host one at a time
    e2e = None
    if not args.no_e2e:
        # results into host memory: the host link, not the kernels, bounds the
        # step, and queries run one after another start the first result's copy
        # earlier than a shared group does (measured), so no type mixing here
        if groups:
            ctx.set_tuning("group_mix", 0)
        hosts = [torch.empty((q.win_len, log.V), dtype=torch.int32, pin_memory=True) for q in qs]
        hspecs = [(q.type, q.source, q.win_begin, q.win_len, h) for q, h in zip(qs, hosts)]
        assert svv.svv_query_batch(ctx.h, hspecs) == [0] * len(qs)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            svv.svv_query_batch(ctx.h, hspecs)
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, world, f"cuda:{dev}")
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for q, h in zip(qs, hosts):
                ctx.query_host(q.type, q.source, q.win_begin, q.win_len, h.numpy())
        dt1 = max_over_ranks(time.perf_counter() - t0, world, f"cuda:{dev}")
        import ctypes
        e2e = {"value": values_per_step * args.steps * world / dt, "unit": UNIT,
               "h2d_bytes_per_step": len(qs) * ctypes.sizeof(svv.svv_query_spec),
               "d2h_bytes_per_step": int(sum(q.win_len * log.V * 4 for q in qs)),
               "inputs": "the step's query arguments (svv_query_spec); the graph stays resident on the device",
               "api": "svv_query_batch, pinned host outputs, one query after another (each result copied "
                      "back while the next computes)",
               "one_at_a_time": {"value": values_per_step * args.steps * world / dt1, "api": "svv_query_host"}}

    if rank == 0:
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peaks = json.load(f)
        except Exception:
            pass
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
        # every phase's roofline: algorithmic bytes per launch (the hot-path
        # table's per-unit figures, and separately the resident layout's
        # floor) over the phase's average event-timed duration
        nlaunch = nphase * len(qs)
        grouped = [q for q in qs if not _isolated(log, q.source)]
        phases = []
        for ph in ("cap", "cup", "qrs", "relax", "scatter"):
            if groups and ph in ("cap", "cup") and len(grouped) > 1:
                # one group launch solves every query of the step: its
                # algorithmic bytes are the member queries' (one unit each),
                # its floor reads the graph once for all of them
                ms = group_ms[ph] / nphase
                sb = sum(algorithmic_bytes(ph, gc, None, q.win_len) for q in grouped)
                lb = group_layout_bytes(ph, gc, len(grouped))
                kname, tkey = GROUP_KERNELS[ph], "group_" + ph
            else:
                ms = phase_ms[ph] / nlaunch
                sb = sum(algorithmic_bytes(ph, gc, st, q.win_len) for sts in all_stats for st, q in zip(sts, qs)) / nlaunch
                lb = sum(layout_bytes(ph, gc, st, q.win_len) for sts in all_stats for st, q in zip(sts, qs)) / nlaunch
                kname, tkey = PHASE_KERNELS[ph], ph
            a = sb / (ms / 1e3) / 1e9 if ms > 0 else 0.0
            al = lb / (ms / 1e3) / 1e9 if ms > 0 else 0.0
            phases.append({"phase": ph, "kernel": kname, "avg_launch_ms": ms, "traffic_key": tkey,
                           "algorithmic_bytes_per_launch": sb, "achieved": a, "frac": a / hbm_peak,
                           "layout_floor": {"bytes_per_launch": lb, "achieved": al, "frac": al / hbm_peak}})
        dom = max(phases, key=lambda p: p["avg_launch_ms"])
        if groups and len(grouped) > 1:
            ph_step = {k: (group_ms[k] / nphase if k in group_ms else v / nphase) for k, v in phase_ms.items()}
            # lane words, two group solves, split; per member extraction,
            # relaxation and scatter, or for a pair of one window length one
            # extraction, one relaxation and two scatters
            pair = len(grouped) == 2 and grouped[0].win_len == grouped[1].win_len and grouped[0].win_len <= 128
            launches = len(qs) - len(grouped) + 4 + (4 if pair else 3 * len(grouped))
            api = ("svv_query_batch: the step's queries in one call, one query group of mixed types "
                   "(batch_mode 2, group_mix 1); the call returns after the step")
        else:
            ph_step = {k: v / nphase for k, v in phase_ms.items()}
            launches = sum(1 if _isolated(log, q.source) else 5 for q in qs)
            api = "svv_query_async per query, one stream, no host wait inside a step"
        last = all_stats[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": desc, "queries_per_step": len(qs), "l2": "flushed between steps (512 MB write)",
                       "api": api,
                       "parallelism": f"replicas x{world}", "tuning": dict(kv.split("=", 1) for kv in args.tune)},
            "roofline": {"bound": "hbm", "kernel": dom["kernel"], "phase": dom["phase"],
                         "achieved": dom["achieved"], "peak": hbm_peak,
                         "peak_source": peak_src + " (copy bandwidth, burst)", "unit": "GB/s", "frac": dom["frac"],
                         "algorithmic_bytes_per_launch": dom["algorithmic_bytes_per_launch"],
                         "avg_launch_ms": dom["avg_launch_ms"],
                         "traffic": recorded_traffic(dom["traffic_key"], args.workload),
                         "layout_floor": dom["layout_floor"]},
            "roofline_phases": phases,
            "phase_ms_per_step": ph_step,
            "plain": plain, "e2e": e2e, "clocks": clocks,
            "gpu_launches": args.steps * launches,
            "query_stats": [{k: v for k, v in st.items() if not k.startswith("ms_")} for st in last],
        }
        if not args.no_cpu_baseline and world == 1:  # timed on the host at N=1 only
            line["cpu_baseline"] = cpu_baseline(log, qs)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
