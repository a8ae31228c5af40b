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
    p.add_argument("--workload", choices=["rmat20", "small"], default="rmat20")
    p.add_argument("--plain-steps", type=int, default=1, help="timed steps of the plain recompute (0 = skip)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--tune", action="append", default=[], metavar="KEY=VALUE",
                   help="library tuning knob (svv_set_tuning), repeatable")
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


def algo_bytes(phase, gc, st, L):
    """Algorithmic bytes of one launch of a phase (the floor each kernel must
    move with the resident layout: 8 B per edge (target, weight), 8 B per mask
    word of an edge not present in every snapshot, 8 B of row offsets and 4 B
    of value per vertex)."""
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


KERNEL_SOURCES = {"cap": ["svv_solve.cu", "svv_device.cuh", "svv_push.cuh", "svv_internal.h"]}


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, only while the
    kernel's sources still hash to the version that was captured."""
    import hashlib
    import re
    if workload != "rmat20" or kernel not in KERNEL_SOURCES:
        return None
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2502_10579_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    try:
        with open(os.path.join(ROOT, "profiles", "solve_kernel_rmat20.md")) as fh:
            for line in fh:
                m = re.match(r"traffic: kernel=(\w+) bytes_per_launch=(\d+) sources_sha256=(\w+)", line.strip())
                if m and m.group(1) == kernel and m.group(3) == h.hexdigest():
                    return int(m.group(2))
    except OSError:
        pass
    return None


def cpu_baseline(log, qs, nthreads=0, snaps=None):
    import oracle
    cores = nthreads or os.cpu_count() or 1
    k = snaps or max(2, min(log.S, cores // len(qs) if cores >= len(qs) else 1))
    t0 = time.perf_counter()
    vals = 0
    for q in qs:
        oracle.query(log, q.type, q.source, q.win_begin, k, nthreads=cores)
        vals += k * log.V
    dt = time.perf_counter() - t0
    return {"value": vals / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(qs)} queries x {k} snapshots (of {qs[0].win_len}) from scratch, "
                      f"threads over snapshots, {dt:.2f} s wall"}


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
        cb = cpu_baseline(log, qs, cores, k)
        times.append(time.perf_counter() - t0)
        vals += len(qs) * k * log.V
    total = sum(times)
    value = vals / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": desc, "sample_snapshots": k},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)

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
    ctx.load_csr(log.V, log.S, rp, col, w, mask)
    ctx.set_tuning("phase_timing", 1)
    for kv in args.tune:
        k, v = kv.split("=", 1)
        ctx.set_tuning(k, int(v))
    outs = [ctx.empty_out(q.win_len) for q in qs]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)

    def step(plain=False):
        sts = []
        for q, o in zip(qs, outs):
            ctx.query(q.type, q.source, q.win_begin, q.win_len, out=o, stream=stream, plain=plain)
            sts.append(ctx.stats())
        return sts

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()

    sampler = ClockSampler(gpu_id_of(dev)) if (rank == 0 and not args.no_clocks) else None
    if sampler:
        sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    phase_ms = {k: 0.0 for k in ("cap", "cup", "qrs", "relax", "scatter")}
    all_stats = []
    for i in range(args.steps):
        starts[i].record(stream)
        sts = step()
        ends[i].record(stream)
        flush.zero_()  # L2 flush between timed steps, outside the event pair
        for st in sts:
            for k in phase_ms:
                phase_ms[k] += st["ms_" + k]
        all_stats.append(sts)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    ms_total = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms_total = max_over_ranks(ms_total, world, f"cuda:{dev}")
    values_per_step = sum(q.win_len * log.V for q in qs)
    value = values_per_step * args.steps * world / (ms_total / 1e3)

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
        plain = {"value": pvalue, "unit": UNIT, "ms_per_step": pms / args.plain_steps,
                 "iu_speedup": value / pvalue}

    # end to end through the public API with host output buffers
    e2e = None
    if not args.no_e2e:
        hosts = [torch.empty((q.win_len, log.V), dtype=torch.int32, pin_memory=True) for q in qs]
        for q, h in zip(qs, hosts):
            ctx.query_host(q.type, q.source, q.win_begin, q.win_len, h.numpy())
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for q, h in zip(qs, hosts):
                ctx.query_host(q.type, q.source, q.win_begin, q.win_len, h.numpy())
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, world, f"cuda:{dev}")
        e2e = {"value": values_per_step * args.steps * world / dt, "unit": UNIT, "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": int(sum(q.win_len * log.V * 4 for q in qs))}

    if rank == 0:
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peaks = json.load(f)
        except Exception:
            pass
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
        # dominant phase and its roofline
        dom = max(phase_ms, key=phase_ms.get)
        nlaunch = args.steps * len(qs)
        abytes = sum(algo_bytes(dom, gc, st, q.win_len) for sts in all_stats for st, q in zip(sts, qs))
        dur_s = phase_ms[dom] / 1e3
        achieved = abytes / dur_s / 1e9 if dur_s > 0 else 0.0
        last = all_stats[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": desc, "queries_per_step": len(qs), "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{world}", "tuning": dict(kv.split("=", 1) for kv in args.tune)},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak,
                         "peak_source": peak_src, "unit": "GB/s", "frac": achieved / hbm_peak,
                         "algorithmic_bytes_per_launch": abytes / nlaunch,
                         "avg_launch_ms": phase_ms[dom] / nlaunch,
                         "traffic": recorded_traffic(dom, args.workload)},
            "phase_ms_per_step": {k: v / args.steps for k, v in phase_ms.items()},
            "plain": plain, "e2e": e2e, "clocks": clocks,
            "gpu_launches": args.steps * len(qs) * 5,
            "query_stats": [{k: v for k, v in st.items() if not k.startswith("ms_")} for st in last],
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(log, qs)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
