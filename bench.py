#!/usr/bin/env python
"""Throughput of exact h-motif / 3h-motif counting (MoCHy-E) on one GB300.

Workload: the seeded medium hypergraph (100,000 nodes, 200,000 distinct
hyperedges, sizes from a truncated power law with exponent 2.5 on [2, 25],
members by Zipf(1.0) popularity, seed 1).  One step is the whole exact path
through the C ABI: load (validation, sorting, duplicate removal, incidence
lists), line-graph projection, exact counting of all 26 h-motifs and 431
3h-motifs.  The metric is hyperedge triples classified per second: the number
of connected hyperedge triples (all instances of all motifs) per step divided
by the step time.

value: inputs already resident in device memory, CUDA events on the
library's stream around K steps.  e2e: the same metric through mochy_load
from pinned host buffers (host-to-device copy inside the timed region) and a
device-to-host read of the counts.  roofline: the dominant kernel's duration
is taken live from the library's traced CUDA events.  cpu_baseline: the
single-threaded CPU oracle on a seeded anchor sample of the same hypergraph.

Multi-GPU (torchrun): every rank counts its own independently seeded
hypergraph of the same shape (weak scaling, no collective on the data path).
`--impl reference` times the CPU oracle instead, on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "hyperedge triples classified/s (exact)"
UNIT = "triples/s"


def _spec(workload: str, seed_offset: int):
    from paper_2310_15668_gb300 import synth
    import dataclasses
    base = {"medium": synth.MEDIUM, "tiny": synth.TINY}[workload]
    return dataclasses.replace(base, seed=base.seed + seed_offset)


def _workload_name(spec) -> str:
    return f"medium exact h/3h-motif counts: {spec.describe()}"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cpu_baseline(off, nodes, n_nodes, seconds: float, seed: int = 12345):
    """Oracle (single thread) on a seeded anchor sample of the workload."""
    import oracle
    E = off.size - 1
    deg_v = np.bincount(nodes, minlength=n_nodes).astype(np.int64)
    bound = np.add.reduceat(deg_v[nodes] - 1, off[:-1]) if E else np.zeros(0, np.int64)
    rng = np.random.default_rng(seed)
    order = rng.permutation(E)
    # anchors drawn uniformly (seeded), skipping hub-containing ones whose
    # neighbourhood bound exceeds 4,000 (one such anchor alone costs minutes)
    cap = 4_000
    cand = [int(i) for i in order if bound[i] <= cap][:20000]
    done_inst, done_time, used, k = 0, 0.0, 0, 0
    step = 1
    while done_time < seconds and k < len(cand):
        anchors = np.array(cand[k:k + step], np.int32)
        k += step
        t = time.perf_counter()
        h, _ = oracle.count_exact_subset(off, nodes, anchors)
        dt = time.perf_counter() - t
        done_inst += int(h.sum())
        done_time += dt
        used += anchors.size
        step = min(step * 2, 512)
    return {"value": done_inst / done_time if done_time > 0 else None, "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": f"{used} anchors drawn uniformly by seed {seed} among hyperedges whose "
                      f"neighbourhood bound is at most {cap} ({done_inst} triples in "
                      f"{done_time:.1f} s, oracle set-up excluded)"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    spec = _spec(args.workload, 0)
    from paper_2310_15668_gb300 import synth
    import oracle
    oracle.build()
    off, nodes = synth.generate(spec)
    per_step = max(args.reference_seconds, 1.0)
    for _ in range(args.warmup):
        _cpu_baseline(off, nodes, spec.n_nodes, per_step / 4, seed=999)
    vals, times = [], []
    t0 = time.perf_counter()
    for s in range(args.steps):
        r = _cpu_baseline(off, nodes, spec.n_nodes, per_step, seed=1000 + s)
        vals.append(r["value"])
    elapsed = time.perf_counter() - t0
    value = float(np.mean(vals))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": _workload_name(spec), "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_15668_gb300 import binding as B, synth
    spec = _spec(args.workload, rank)
    off, nodes = synth.generate(spec)
    d_off = torch.from_numpy(off).cuda()
    d_nodes = torch.from_numpy(nodes).cuda()
    ctx = B.Context(device=local)
    stream = torch.cuda.ExternalStream(ctx.stream, device=local)
    instances = 0

    def step(trace=False):
        nonlocal instances
        B.mochy_load_device(ctx.h, spec.n_nodes, off.size - 1, d_off.data_ptr(),
                            d_nodes.data_ptr())
        ctx.project()
        h, h3 = ctx.count_exact()
        instances = int(h.sum())
        return h, h3

    for _ in range(args.warmup):
        step()
    B.mochy_trace(ctx.h, 1)            # phase events only: no effect on the kernels
    phases = []
    launches0 = B.mochy_kernel_launches()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        start.record(stream)
        for _ in range(args.steps):
            step()
            phases.append(B.mochy_trace_read(ctx.h))
        end.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches = B.mochy_kernel_launches() - launches0
    ms = start.elapsed_time(end)
    B.mochy_trace(ctx.h, 0)
    t_max = torch.tensor([ms], dtype=torch.float64, device="cuda")
    total = torch.tensor([float(instances) * args.steps], dtype=torch.float64, device="cuda")
    if ws > 1:
        torch.distributed.all_reduce(t_max, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(total)
    ms_max = float(t_max.item())
    value = float(total.item()) / (ms_max / 1000.0)

    # kernel statistics (scanned words) from one more, untimed step at trace level 2
    B.mochy_trace(ctx.h, 2)
    step()
    stats_trace = B.mochy_trace_read(ctx.h)
    B.mochy_trace(ctx.h, 0)

    # end to end through the public API from pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        p_off = torch.from_numpy(off).pin_memory().numpy()
        p_nodes = torch.from_numpy(nodes).pin_memory().numpy()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.e2e_steps):
            ctx.load(spec.n_nodes, p_off, p_nodes)
            ctx.project()
            h, _ = ctx.count_exact()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        e2e = {"value": float(h.sum()) * args.e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(p_off.nbytes + p_nodes.nbytes),
               "d2h_bytes_per_step": 457 * 8}

    if rank != 0:
        ctx.close()
        return 0
    # roofline of the dominant kernel, from the traced events of the timed steps
    peak, peak_kind = _peaks()
    keys = set().union(*(p["phases_ms"].keys() for p in phases)) if phases else set()
    avg = {k: float(np.mean([p["phases_ms"].get(k, 0.0) for p in phases])) for k in keys}
    dom = max(avg, key=avg.get) if avg else None
    st = stats_trace
    roof = None
    if dom == "dense triangles" and avg[dom] > 0:
        # algorithmic bytes: every scanned word reads one word of the partner
        # row's bitmap, four size planes, and the words of the bitmaps of the
        # heavy nodes of e_a | e_b (about two per word on this workload)
        words = float(st.get("words_scanned", 0))
        algo = words * 4.0 * (1 + 4 + 2)
        achieved = algo / (avg[dom] / 1000.0) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": "k_dense_triangles",
                "kernel_ms": avg[dom], "peak_kind": peak_kind}
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = _cpu_baseline(off, nodes, spec.n_nodes, args.cpu_seconds)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": _workload_name(spec), "triples_per_step": instances,
                       "l2": "inputs larger than L2 (line graph of 30 GB per step)",
                       "parallelism": f"independent hypergraph per rank x{ws}"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk.summary(), "phases_ms": avg, "trace": st}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=["medium", "tiny"], default="medium")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--reference-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
