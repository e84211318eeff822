"""Run one traced exact count on a seeded synthetic hypergraph.

    python -m paper_2310_15668_gb300.count_case --edges 10000 --dense-threshold 256

The hypergraph has N = E/2 nodes, sizes from a truncated power law with
exponent 2.5 on [2, 25] and Zipf(1.0) members (seed 5 unless given).  Prints
the number of instances and the trace of the call (phase times, dense rows,
scanned words) as one JSON line.  Useful as a small, self-contained case for
profilers.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--edges", type=int, default=10000)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--dense-threshold", type=int, default=0)
    ap.add_argument("--trace", type=int, default=2)
    a = ap.parse_args(argv)
    from paper_2310_15668_gb300 import binding as B, synth
    spec = synth.HypergraphSpec(max(a.edges // 2, 64), a.edges, 2, 25, "powerlaw", 2.5, "zipf", 1.0,
                                seed=a.seed)
    off, nodes = synth.generate(spec)
    with B.Context(dense_threshold=a.dense_threshold) as c:
        c.load(spec.n_nodes, off, nodes)
        n_w, max_deg = c.project()
        B.mochy_trace(c.h, a.trace)
        h, _ = c.count_exact()
        out = {"hypergraph": spec.describe(), "hyperwedges": n_w, "max_line_degree": max_deg,
               "instances": int(h.sum()), "trace": B.mochy_trace_read(c.h)}
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
