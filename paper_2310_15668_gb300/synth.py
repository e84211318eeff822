"""Seeded synthetic hypergraphs that stand in for the paper's datasets.

This module only draws inputs.  It holds none of the counting method's
arithmetic and is shared by the oracle tests, the GPU tests and the bench.

The paper's datasets (Section 5.1, Table "dataset_table") are not available,
so every workload is a seeded synthetic hypergraph with the shapes of that
table: hyperedge sizes up to 25, heavy-tailed node degrees, hub-dominated
line graphs.

Recipe (every draw comes from a counter-based SplitMix64 stream, so the same
seed gives the same hypergraph on every machine and numpy version):

* hyperedge size: a discrete distribution on [s_min, s_max], either uniform
  or a truncated power law P(s) ~ s^-alpha;
* members: ``size`` distinct nodes drawn one after another from a node
  popularity distribution (uniform, or Zipf P(rank r) ~ r^-z with rank r
  mapped to node id r-1); a draw that repeats a node already in the
  hyperedge is redrawn, which is the same law as drawing without replacement
  with the weights renormalised over the remaining nodes;
* candidates are drawn until ``n_edges`` distinct hyperedges exist;
  duplicates are dropped, the first occurrence is kept, and hyperedges keep
  their order of first occurrence.  Node lists are sorted ascending.

The output is a CSR pair ``(offsets int64[E+1], nodes int32[sum |e|])``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied elementwise to uint64 counters."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    k = np.array([(seed * 0x100000001B3 + stream * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF],
                 dtype=np.uint64)
    return _splitmix64(_splitmix64(k))[0]


def _uniform01(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the 53 high bits of SplitMix64."""
    key = _stream_key(seed, stream)
    with np.errstate(over="ignore"):
        u = _splitmix64((counters.astype(np.uint64) + key) & _M64)
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass(frozen=True)
class HypergraphSpec:
    """Parameters of one synthetic hypergraph."""
    n_nodes: int
    n_edges: int
    s_min: int = 2
    s_max: int = 25
    size_law: str = "powerlaw"      # "uniform" or "powerlaw"
    size_alpha: float = 2.5
    member_law: str = "zipf"        # "uniform" or "zipf"
    zipf_s: float = 1.0
    seed: int = 0

    def describe(self) -> str:
        size = (f"U[{self.s_min},{self.s_max}]" if self.size_law == "uniform"
                else f"s^-{self.size_alpha} on [{self.s_min},{self.s_max}]")
        mem = "uniform" if self.member_law == "uniform" else f"Zipf({self.zipf_s})"
        return (f"N={self.n_nodes} E={self.n_edges} sizes {size} members {mem} "
                f"seed {self.seed}")


# The seeded workloads (sizes, laws and seeds of the benchmark configurations).
TINY = HypergraphSpec(1000, 2000, 2, 5, "uniform", 0.0, "uniform", 0.0, seed=0)
MEDIUM = HypergraphSpec(100_000, 200_000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=1)
LARGE = HypergraphSpec(1_500_000, 2_500_000, 2, 25, "powerlaw", 2.2, "zipf", 1.1, seed=2)


def _cdf(weights: np.ndarray) -> np.ndarray:
    c = np.cumsum(weights, dtype=np.float64)
    c /= c[-1]
    c[-1] = 1.0
    return c


def _size_cdf(spec: HypergraphSpec) -> np.ndarray:
    s = np.arange(spec.s_min, spec.s_max + 1, dtype=np.float64)
    if spec.size_law == "uniform":
        w = np.ones_like(s)
    else:
        w = s ** (-float(spec.size_alpha))
    return _cdf(w)


def _node_cdf(spec: HypergraphSpec) -> np.ndarray:
    if spec.member_law == "uniform":
        return _cdf(np.ones(spec.n_nodes, dtype=np.float64))
    r = np.arange(1, spec.n_nodes + 1, dtype=np.float64)
    return _cdf(r ** (-float(spec.zipf_s)))


def _draw_members(spec, node_cdf, sizes, cand_ids, rnd):
    """First ``sizes[r]`` distinct nodes of each row's draw sequence."""
    width = 2 * spec.s_max + 8
    slots = np.arange(width, dtype=np.uint64)
    ctr = (cand_ids.astype(np.uint64)[:, None] * np.uint64(1 << 12)
           + np.uint64(rnd * width) + slots[None, :])
    u = _uniform01(spec.seed, 2, ctr)
    draws = np.searchsorted(node_cdf, u, side="right").astype(np.int64)
    np.minimum(draws, spec.n_nodes - 1, out=draws)
    order = np.argsort(draws, axis=1, kind="stable")
    sd = np.take_along_axis(draws, order, axis=1)
    dup_sorted = np.zeros_like(sd, dtype=bool)
    dup_sorted[:, 1:] = sd[:, 1:] == sd[:, :-1]
    first = np.empty_like(dup_sorted)
    np.put_along_axis(first, order, ~dup_sorted, axis=1)
    rank = np.cumsum(first, axis=1)
    take = first & (rank <= sizes[:, None])
    ok = rank[:, -1] >= sizes
    return draws, take, ok


def generate(spec: HypergraphSpec, max_rounds: int = 64):
    """Return ``(offsets, nodes)``: ``spec.n_edges`` distinct hyperedges."""
    size_cdf = _size_cdf(spec)
    node_cdf = _node_cdf(spec)
    if spec.s_max > spec.n_nodes:
        raise ValueError("s_max exceeds the node count")
    keys_seen: dict = {}
    rows: list = []
    next_cand = 0
    need = spec.n_edges
    while len(rows) < need:
        batch = max(1024, int((need - len(rows)) * 1.05) + 64)
        cand = np.arange(next_cand, next_cand + batch, dtype=np.int64)
        next_cand += batch
        u = _uniform01(spec.seed, 1, cand)
        sizes = spec.s_min + np.searchsorted(size_cdf, u, side="right")
        sizes = np.minimum(sizes, spec.s_max).astype(np.int64)
        out = np.full((batch, spec.s_max), np.iinfo(np.int64).max, dtype=np.int64)
        todo = np.arange(batch)
        for rnd in range(max_rounds):
            if todo.size == 0:
                break
            draws, take, ok = _draw_members(spec, node_cdf, sizes[todo], cand[todo], rnd)
            okr = np.nonzero(ok)[0]
            if okr.size:
                t = take[okr]
                d = draws[okr]
                cnt = t.sum(axis=1)
                vals = d[t]
                rr = np.repeat(np.arange(okr.size), cnt)
                cc = np.arange(vals.size) - np.repeat(np.cumsum(cnt) - cnt, cnt)
                sub = np.full((okr.size, spec.s_max), np.iinfo(np.int64).max, dtype=np.int64)
                sub[rr, cc] = vals
                out[todo[okr]] = sub
            todo = todo[~ok]
        if todo.size:
            raise RuntimeError("member draws did not converge")
        out.sort(axis=1)
        view = np.ascontiguousarray(out).view(np.dtype((np.void, 8 * spec.s_max))).ravel()
        for r in range(batch):
            k = view[r].tobytes()
            if k in keys_seen:
                continue
            keys_seen[k] = len(rows)
            rows.append(out[r, :sizes[r]])
            if len(rows) == need:
                break
    sizes = np.fromiter((len(r) for r in rows), dtype=np.int64, count=len(rows))
    offsets = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    nodes = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    return offsets, nodes


def loguniform_edges(seed: int, index: int, lo: int, hi: int) -> int:
    """Hyperedge count of the ``index``-th graph of a batch, log-uniform in [lo, hi]."""
    u = float(_uniform01(seed, 7, np.array([index], dtype=np.int64))[0])
    return int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))))


def batch_spec(seed: int, index: int, lo: int, hi: int, alpha: float = 2.5,
               zipf_s: float = 1.0) -> HypergraphSpec:
    """One member of a batch of graphs: E log-uniform in [lo, hi], N = E/2."""
    e = loguniform_edges(seed, index, lo, hi)
    return HypergraphSpec(max(e // 2, 64), e, 2, 25, "powerlaw", alpha, "zipf", zipf_s,
                          seed=seed * 1_000_003 + index)


def plant_cluster(offsets, nodes, n_extra: int, pool_lo: int, pool_size: int, s_lo: int,
                  s_hi: int, seed: int):
    """Append ``n_extra`` hyperedges drawn from a small pool of nodes.

    Each new hyperedge has a size uniform in [s_lo, s_hi] and takes that many
    distinct nodes of the pool [pool_lo, pool_lo + pool_size) (the nodes with
    the smallest keys of one SplitMix64 draw per pool node).  Hyperedges drawn
    from one small pool overlap heavily with each other, which the Zipf and
    uniform laws above almost never produce.  Returns ``(offsets, nodes)`` of
    the input followed by the new hyperedges (repeats are left in; loading a
    hypergraph drops them)."""
    off = np.asarray(offsets, dtype=np.int64)
    nod = np.asarray(nodes, dtype=np.int32)
    ids = np.arange(n_extra, dtype=np.int64)
    u = _uniform01(seed, 9, ids)
    sizes = s_lo + np.minimum((u * (s_hi - s_lo + 1)).astype(np.int64), s_hi - s_lo)
    ctr = ids[:, None] * np.int64(1 << 16) + np.arange(pool_size, dtype=np.int64)[None, :]
    keys = _uniform01(seed, 10, ctr.ravel()).reshape(n_extra, pool_size)
    order = np.argsort(keys, axis=1, kind="stable")
    rows = [np.sort(order[r, :sizes[r]]) + pool_lo for r in range(n_extra)]
    new_off = np.zeros(n_extra + 1, dtype=np.int64)
    np.cumsum(sizes, out=new_off[1:])
    out_off = np.concatenate([off, off[-1] + new_off[1:]])
    out_nodes = np.concatenate([nod] + [r.astype(np.int32) for r in rows]) if n_extra else nod
    return out_off, out_nodes
