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
CPU oracle (its anchor loop on every host core) on a seeded anchor sample of
the same hypergraph.  sampled: candidates classified/s of MoCHy-A+ with
r = 2,000,000 hyperwedges on the same projected hypergraph.  onthefly (rank
0, one GPU): MoCHy-A+ without the line graph on the large workload (1.5M
nodes, 2.5M hyperedges, Zipf(1.1), seed 2; its line graph would need 6 to
12 TB), r = 2,000,000.

batch (rank 0, one GPU): significance and CP of 16 seeded hypergraphs (E
log-uniform in [2,000, 20,000], N = E/2, power-law sizes on [2, 25], Zipf(1.0)
members), each against 32 randomized copies: CPs/s of mochy_profile_batch
(all 528 hypergraphs generated on the device and counted in one CUDA-graph
launch) beside CPs/s of mochy_profile called once per hypergraph, with the
check that both give identical counts and CPs.

serving (rank 0, one GPU): a Poisson stream of count and CP requests
(E log-uniform in [1,000, 4,000] from a pool of seeded hypergraphs; 90%
exact counts, 10% profiles with 4 copies) offered at 200/s to a
mochy_server with 8 slots and a 120 GB budget; p50/p99 latency and
completed requests/s.

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


WORKLOADS = ("medium", "tiny", "zipf10k", "zipf40k")

# DRAM bytes (read + write) of one k_dense_triangles launch, measured with
# ncu (dram__bytes_read.sum + dram__bytes_write.sum, one pass) on the
# workload and threshold named, for the kernel as it is now; reported as
# null for any other workload or threshold, and emptied whenever the kernel
# changes until it is measured again.
DENSE_TRAFFIC = {("medium", 1024): 8.640e12}


def _spec(workload: str, seed_offset: int):
    """The bench workload (medium) or a smaller case of the same shape for
    profilers (zipf10k, zipf40k: N = E/2, sizes s^-2.5 on [2, 25], Zipf(1.0)
    members, seed 5)."""
    from paper_2310_15668_gb300 import synth
    import dataclasses
    base = {"medium": synth.MEDIUM, "tiny": synth.TINY,
            "zipf10k": synth.HypergraphSpec(5000, 10000, 2, 25, "powerlaw", 2.5, "zipf", 1.0,
                                            seed=5),
            "zipf40k": synth.HypergraphSpec(20000, 40000, 2, 25, "powerlaw", 2.5, "zipf", 1.0,
                                            seed=5)}[workload]
    return dataclasses.replace(base, seed=base.seed + seed_offset)


def _workload_name(spec) -> str:
    return f"exact h/3h-motif counts: {spec.describe()}"


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


def reduce_over_ranks(ms: float, units: float, world_size: int, device: str):
    """Whole-job timing over ranks: the slowest rank's time and the work of
    all ranks (each rank counts its own hypergraph; no data-path exchange)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    if world_size > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u)
    return float(t.item()), float(u.item())


def partition_rows(deg, world_size: int):
    """Rows of one hypergraph dealt to ranks for the row-sharded count: rows in
    decreasing estimated work |N_e|^2 (pairs of neighbours), dealt in snake
    order (0, 1, .., n-1, n-1, .., 0, ...), so every rank gets a similar share
    of the heavy rows.  Returns one int32 array of rows per rank."""
    deg = np.asarray(deg, dtype=np.int64)
    order = np.lexsort((np.arange(deg.size), -(deg * deg)))
    pos = np.arange(order.size)
    lap, k = pos // world_size, pos % world_size
    owner = np.where(lap % 2 == 0, k, world_size - 1 - k)
    return [np.sort(order[owner == r]).astype(np.int32) for r in range(world_size)]


def reduce_counts(counts, world_size: int, device: str):
    """Sum of every rank's int64 motif histogram (the row-sharded count's one
    exchange; shares may be negative, the sum is the exact count)."""
    import torch
    t = torch.as_tensor(np.ascontiguousarray(counts, dtype=np.int64), device=device)
    if world_size > 1:
        import torch.distributed as dist
        dist.all_reduce(t)
    return t.cpu().numpy()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cpu_baseline(off, nodes, n_nodes, seconds: float, seed: int = 12345, threads: int = 0):
    """The oracle's MoCHy-E (hash sets, the paper's hyperedge-centric loop)
    on a seeded anchor sample of the workload, its anchor loop on `threads`
    host threads (0 = every core this process may use)."""
    import oracle
    nt = oracle.host_threads() if threads == 0 else threads
    E = off.size - 1
    deg_v = np.bincount(nodes, minlength=n_nodes).astype(np.int64)
    bound = np.add.reduceat(deg_v[nodes] - 1, off[:-1]) if E else np.zeros(0, np.int64)
    rng = np.random.default_rng(seed)
    order = rng.permutation(E)
    # anchors drawn uniformly (seeded), skipping hub-containing ones whose
    # neighbourhood bound exceeds 4,000 (one such anchor alone costs minutes)
    cap = 4_000
    cand = [int(i) for i in order if bound[i] <= cap][:40000]
    # every oracle call first builds its hash sets: timed once with no anchor
    # and taken off each call's time
    t = time.perf_counter()
    oracle.count_exact_ranked(off, nodes, np.zeros(0, np.int32), None, threads=nt)
    setup = time.perf_counter() - t
    done_inst, done_time, used, k = 0, 0.0, 0, 0
    step = nt
    while done_time < seconds and k < len(cand):
        anchors = np.array(cand[k:k + step], np.int32)
        k += step
        t = time.perf_counter()
        h, _ = oracle.count_exact_ranked(off, nodes, anchors, None, threads=nt)
        dt = max(time.perf_counter() - t - setup, 1e-6)
        done_inst += int(h.sum())
        done_time += dt
        used += anchors.size
        step = min(step * 2, 1024 * nt)
    return {"value": done_inst / done_time if done_time > 0 else None, "unit": UNIT, "cores": nt,
            "kind": "oracle",
            "sample": f"{used} anchors drawn uniformly by seed {seed} among hyperedges whose "
                      f"neighbourhood bound is at most {cap} ({done_inst} triples in "
                      f"{done_time:.1f} s on {nt} host threads, oracle set-up excluded)"}


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
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _sampled_measure(ctx, args):
    """Candidates classified per second by MoCHy-A+ (Algorithm
    "sampling_ver2") on the projected workload: r hyperwedges drawn with
    Philox, every hyperedge adjacent to either end classified.  Device time
    with CUDA events on the library's stream, after one warm-up call."""
    import torch
    from paper_2310_15668_gb300 import binding as B
    stream = torch.cuda.ExternalStream(ctx.stream)
    r = int(args.sampled_r)
    ctx.count_sampled(B.MOCHY_A_PLUS, r, 1)
    times, cands = [], 0
    for k in range(args.sampled_steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        raw_h, _, _, _ = ctx.count_sampled(B.MOCHY_A_PLUS, r, 2 + k)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        cands = int(raw_h.sum())
    ms = float(np.mean(times))
    return {"metric": "candidates classified/s (MoCHy-A+)", "value": cands / (ms / 1000.0),
            "unit": "candidates/s", "r": r, "candidates_per_call": cands, "ms_per_call": ms,
            "calls": args.sampled_steps}


def _onthefly_measure(args):
    """MoCHy-A+ without the line graph on the large workload (1.5M nodes,
    2.5M hyperedges, sizes s^-2.2 on [2, 25], Zipf(1.1) members, seed 2):
    r = 2,000,000 hyperwedges drawn by Philox seed 2.  Its line graph (4e11
    to 8e11 hyperwedges) does not fit in device memory.  The first call
    after the load builds the membership bitmaps and the line-graph degrees
    (reported as set-up); the timed calls classify r draws each.  Device
    time with CUDA events on the library's stream."""
    import torch
    from paper_2310_15668_gb300 import binding as B, synth
    spec = synth.LARGE if args.onthefly_workload == "large" else _spec(args.onthefly_workload, 0)
    t = time.perf_counter()
    off, nodes = synth.generate(spec)
    gen_s = time.perf_counter() - t
    r = int(args.onthefly_r)
    with B.Context() as c:
        stream = torch.cuda.ExternalStream(c.stream)
        c.load(spec.n_nodes, off, nodes)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        first = c.count_sampled_onthefly(1, 2)
        e1.record(stream)
        torch.cuda.synchronize()
        setup_ms = e0.elapsed_time(e1)
        times, cands = [], 0
        for k in range(args.sampled_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            raw_h, _, est_h, _, nw = c.count_sampled_onthefly(r, 2 + k)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            cands = int(raw_h.sum())
        B.mochy_trace(c.h, 2)
        c.count_sampled_onthefly(r, 2)
        tr = B.mochy_trace_read(c.h)
    ms = float(np.mean(times))
    return {"metric": "candidates classified/s (MoCHy-A+ without the line graph)",
            "value": cands / (ms / 1000.0), "unit": "candidates/s", "r": r,
            "candidates_per_call": cands, "ms_per_call": ms, "calls": args.sampled_steps,
            "setup_ms": setup_ms, "hyperwedges": int(first[4]),
            "config": {"workload": f"{args.onthefly_workload}: {spec.describe()}, r = {r} "
                                   f"hyperwedges by Philox seed 2 (+ call index)",
                       "line_graph_bytes_if_projected": int(first[4]) * 16},
            "generate_s": gen_s,
            "trace": {k: tr.get(k) for k in ("otf_candidates", "otf_words", "otf_list_entries",
                                             "otf_exact", "otf_bitmaps")}}


def _extensions_measure(args):
    """kh-motifs (k = 4, thresholds 1 and 2), instance enumeration and radial
    node profiles, each one timed call through the C ABI (host results
    included) on a seeded Zipf hypergraph of the medium shape, scaled down:
    their per-instance scans suit hypergraphs of up to about 1e10 triples."""
    from paper_2310_15668_gb300 import binding as B, synth
    out = {}

    def timed(fn):
        fn()                                   # warm-up (tables, allocation)
        t = time.perf_counter()
        r = fn()
        return r, time.perf_counter() - t

    g4 = synth.HypergraphSpec(2000, 4000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=6)
    off, nodes = synth.generate(g4)
    with B.Context() as c:
        c.load(g4.n_nodes, off, nodes)
        c.project()
        (h, kh), dt = timed(lambda: c.count_kh(4, (1, 2)))
        out["kh4"] = {"metric": "instances classified/s into 3,076 4h-motifs", "value":
                      float(h.sum()) / dt, "seconds": dt, "instances": int(h.sum()),
                      "workload": g4.describe()}
    g1 = synth.HypergraphSpec(500, 1000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=3)
    off, nodes = synth.generate(g1)
    with B.Context() as c:
        c.load(g1.n_nodes, off, nodes)
        c.project()
        n_inst = int(c.count_exact()[0].sum())
        (rows, n), dt = timed(lambda: c.enumerate(n_inst))
        out["enumerate"] = {"metric": "instances written/s (i, j, k, h, 3h rows)", "value":
                            n / dt, "seconds": dt, "instances": int(n),
                            "workload": g1.describe()}
        (rh, r3), dt = timed(lambda: c.radial_node_profile())
        out["radial_np"] = {"metric": "radial node profiles/s", "value": g1.n_nodes / dt,
                            "seconds": dt, "nodes": g1.n_nodes, "workload": g1.describe()}
    return out


def _batch_measure(args, lo=None, hi=None):
    """CPs/s of the batched profile against one profile call per hypergraph."""
    from paper_2310_15668_gb300 import binding as B, synth
    G, R = args.batch_graphs, args.batch_copies
    lo = args.batch_lo if lo is None else lo
    hi = args.batch_hi if hi is None else hi
    gs = []
    for i in range(G):
        s = synth.batch_spec(4, i, lo, hi)
        off, nodes = synth.generate(s)
        gs.append((s.n_nodes, off, nodes))
    seeds = [1000 + g for g in range(G)]
    B.mochy_profile_batch(gs[:2], 2, seeds[:2])            # warm-up (library, allocator)
    t = time.perf_counter()
    res = B.mochy_profile_batch(gs, R, seeds)
    t_batch = time.perf_counter() - t
    t = time.perf_counter()
    same = True
    for g, (n, off, nodes) in enumerate(gs):
        with B.Context() as c:
            c.load(n, off, nodes)
            one = c.profile(R, seeds[g])
        same = same and np.array_equal(res[4][g], one["counts_h"]) \
            and np.array_equal(res[5][g], one["counts_3h"]) \
            and np.array_equal(res[1][g], one["cp_h"]) and np.array_equal(res[3][g], one["cp_3h"])
    t_one = time.perf_counter() - t
    info = res[7]
    return {"metric": "CPs/s (significance + characteristic profile)",
            "value": G / t_batch, "one_at_a_time": G / t_one, "speedup": t_one / t_batch,
            "identical_counts_and_cps": bool(same),
            "config": {"workload": f"{G} hypergraphs, E log-uniform in [{lo}, "
                                   f"{hi}], N = E/2, sizes s^-2.5 on [2,25], Zipf(1.0)"
                                   f" members, {R} randomized copies each (scaled-down variant of"
                                   f" E in [50000, 500000])",
                       "hypergraphs_counted": int(info["n_units"]),
                       "triples_counted": int(info["instances"]), "waves": int(info["n_waves"])},
            "batch_s": t_batch, "one_at_a_time_s": t_one,
            "phases_ms": {k: info[k] for k in ("ms_generate", "ms_project", "ms_prepare",
                                               "ms_count", "ms_finish")}}


def _tuner_measure(ctx, st):
    """The measured dense-threshold tuner on the bench hypergraph, after the
    timed steps: each of its candidate thresholds times the dense count of
    the same 2 % row sample with CUDA events, and the fastest is its pick;
    reported beside the threshold the timed steps used."""
    from paper_2310_15668_gb300 import binding as B
    t = time.perf_counter()
    best, tried = B.mochy_tune_dense_threshold(ctx.h)
    return {"kind": "measured (CUDA events on a 2 % row sample per candidate)",
            "threshold_of_timed_steps": int(st.get("dense_threshold", 0)), "best": int(best),
            "candidates_ms": {str(int(thr)): float(ms) for thr, ms in tried},
            "seconds": time.perf_counter() - t}


def _serving_measure(args):
    """Latency and throughput of a Poisson request stream on a mochy_server."""
    import threading
    from paper_2310_15668_gb300 import binding as B, synth
    rng = np.random.default_rng(7)
    pool = []
    for i in range(args.serving_pool):
        s = synth.batch_spec(5, i, 1000, args.serving_hi)
        off, nodes = synth.generate(s)
        pool.append((s.n_nodes, off, nodes))
    n = args.serving_requests
    gaps = rng.exponential(1.0 / args.serving_rate, size=n)
    kinds = rng.random(n) < 1.0 - args.serving_profiles
    picks = rng.integers(0, len(pool), size=n)
    tickets = [0] * n
    with B.Server(n_slots=args.serving_slots, budget=120 << 30) as srv:
        def client():
            t0 = time.perf_counter()
            due = 0.0
            for i in range(n):
                due += gaps[i]
                wait = t0 + due - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                g = pool[picks[i]]
                if kinds[i]:
                    tickets[i] = srv.submit(B.MOCHY_REQ_EXACT, *g)
                else:
                    tickets[i] = srv.submit(B.MOCHY_REQ_PROFILE, *g, n_random=4, seed=i)
        th = threading.Thread(target=client)
        t_start = time.perf_counter()
        th.start()
        th.join()
        t_offered = time.perf_counter() - t_start
        ok = 0
        for t in tickets:
            r = None
            while r is None:
                r = srv.poll(t, wait_ms=1000)
            ok += r["status"] >= 0
        st = srv.stats()
    return {"metric": "request latency p50/p99 (ms) and completed requests/s",
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "requests_per_s": st["throughput_rps"], "offered_per_s": n / t_offered,
            "completed": int(ok), "requests": n, "peak_in_flight": int(st["peak_in_flight"]),
            "config": {"workload": f"{n} requests, Poisson {args.serving_rate}/s, E log-uniform "
                                   f"in [1000, {args.serving_hi}] from {len(pool)} seeded "
                                   f"hypergraphs (scaled-down variant of [1e3, 1e6]), "
                                   f"{100 * (1 - args.serving_profiles):.0f}% exact counts, "
                                   f"{100 * args.serving_profiles:.0f}% profiles with 4 copies",
                       "slots": args.serving_slots, "budget_bytes": 120 << 30}}


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
    # weak scaling: every rank its own hypergraph; --shard-rows: one
    # hypergraph, its rows shared out (strong scaling)
    spec = _spec(args.workload, 0 if args.shard_rows else rank)
    off, nodes = synth.generate(spec)
    d_off = torch.from_numpy(off).cuda()
    d_nodes = torch.from_numpy(nodes).cuda()
    ctx = B.Context(device=local, dense_threshold=args.dense_threshold)
    stream = torch.cuda.ExternalStream(ctx.stream, device=local)
    instances = 0

    shard = args.shard_rows and ws > 1
    my_rows = None

    def step(trace=False):
        nonlocal instances, my_rows
        B.mochy_load_device(ctx.h, spec.n_nodes, off.size - 1, d_off.data_ptr(),
                            d_nodes.data_ptr())
        ctx.project()
        if shard:
            # one hypergraph, rows dealt to ranks; the share of each rank's
            # rows summed over ranks is the exact count
            if my_rows is None:
                my_rows = partition_rows(ctx.line_degrees(), ws)[rank]
            h, h3 = ctx.count_exact_rows(my_rows)
            both = reduce_counts(np.concatenate([h, h3]), ws, "cuda")
            h, h3 = both[:26], both[26:]
        else:
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
    units_here = float(instances) * args.steps
    if shard and rank != 0:
        units_here = 0.0                     # the one hypergraph is counted once
    ms_max, total_units = reduce_over_ranks(ms, units_here, ws, "cuda")
    value = total_units / (ms_max / 1000.0)

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
            if shard:
                h, h3 = ctx.count_exact_rows(my_rows)
                h = reduce_counts(np.concatenate([h, h3]), ws, "cuda")[:26]
            else:
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
        # algorithmic bytes of the classification (candidate stream, 5 B of
        # HBM per classified candidate: a 4-byte hyperedge id and its 1-byte
        # overlap); the candidates the dense kernel classifies per launch are
        # its closed triangles, counted by the traced step
        cand = float(st.get("candidates", 0))
        sec = avg[dom] / 1000.0
        achieved = 5.0 * cand / sec / 1e9
        # the kernel's own loads per scanned word: 16 bytes of row a's overlap
        # planes and adjacency mask, 16 of row b's, 16 of size planes and one
        # bitmap word per heavy node of e_a & e_b
        words = float(st.get("words_scanned", 0))
        hw = float(st.get("dense_hyperwedges", 0)) or 1.0
        n_t = float(st.get("heavy_bitmaps", 0)) / hw
        loads = words * 4.0 * (4 + 4 + 4 + n_t)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": (args.traffic_bytes if args.traffic_bytes is not None else
                            DENSE_TRAFFIC.get((args.workload, int(st.get("dense_threshold", 0))))),
                "kernel": "k_dense_triangles", "kernel_ms": avg[dom], "peak_kind": peak_kind,
                "candidates_per_launch": cand, "bytes_per_candidate": 5,
                "l2_term": {"bytes_per_candidate": 15, "achieved_gbs": 15.0 * cand / sec / 1e9},
                "load_model": {"bytes": loads, "achieved_gbs": loads / sec / 1e9,
                               "frac": loads / sec / 1e9 / peak}}
    sampled = None
    if args.sampled_r > 0:
        sampled = _sampled_measure(ctx, args)
    tuner = None
    if ws == 1 and not shard and not args.no_tuner:
        tuner = _tuner_measure(ctx, st)
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = _cpu_baseline(off, nodes, spec.n_nodes, args.cpu_seconds)
    batch = batch_small = serving = onthefly = extensions = None
    if ws == 1 and not args.no_extras:
        ctx.close()                       # free the medium line graph first
        if args.onthefly_r > 0:
            onthefly = _onthefly_measure(args)
        batch = _batch_measure(args)
        batch_small = _batch_measure(args, 200, 2000)
        serving = _serving_measure(args)
        extensions = _extensions_measure(args)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": _workload_name(spec), "triples_per_step": instances,
                       "l2": "inputs larger than L2 (line graph of 30 GB per step)",
                       "parallelism": (f"rows of one hypergraph over {ws} ranks, one all-reduce "
                                       f"of the 457 int64 bins" if shard else
                                       f"independent hypergraph per rank x{ws}")},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk.summary(), "phases_ms": avg, "trace": st, "sampled": sampled,
            "tuner": tuner,
            "onthefly": onthefly, "batch": batch, "batch_small": batch_small,
            "serving": serving, "extensions": extensions}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="medium")
    ap.add_argument("--dense-threshold", type=int, default=0,
                    help="split kernel threshold (0: the tuner's choice)")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="DRAM bytes per dense-kernel launch from an ncu capture, if known")
    ap.add_argument("--sampled-r", type=int, default=2_000_000,
                    help="MoCHy-A+ samples of the candidates/s line (0: skip)")
    ap.add_argument("--sampled-steps", type=int, default=3)
    ap.add_argument("--shard-rows", action="store_true",
                    help="with several ranks: count one hypergraph with its rows shared out")
    ap.add_argument("--onthefly-r", type=int, default=2_000_000,
                    help="MoCHy-A+ draws on the large workload without a line graph (0: skip)")
    ap.add_argument("--onthefly-workload", choices=["large"] + list(WORKLOADS), default="large")
    ap.add_argument("--only-onthefly", action="store_true",
                    help="run only the MoCHy-A+ measurement without a line graph (a profiler case)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--reference-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tuner", action="store_true",
                    help="skip the measured threshold tuner after the timed steps")
    ap.add_argument("--no-extras", action="store_true", help="skip the batch and serving lines")
    ap.add_argument("--batch-graphs", type=int, default=16)
    ap.add_argument("--batch-copies", type=int, default=32)
    ap.add_argument("--batch-lo", type=int, default=2000)
    ap.add_argument("--batch-hi", type=int, default=20000)
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--serving-hi", type=int, default=4000)
    ap.add_argument("--serving-profiles", type=float, default=0.1)
    ap.add_argument("--serving-pool", type=int, default=64)
    ap.add_argument("--serving-slots", type=int, default=8)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only_onthefly:
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps(_onthefly_measure(args)), flush=True)
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
