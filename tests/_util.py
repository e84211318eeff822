"""Helpers shared by the tests: brute force, micro graphs, canonical tuples.

Everything here is written from the definitions in Section 2 of the paper and
shares no code with the oracle or with the CUDA library.
"""
from __future__ import annotations

import itertools
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_BF_SRC = os.path.join(HERE, "bruteforce.c")
_BF_BIN = os.path.join(HERE, "_build", "bruteforce")


def csr_from_sets(sets):
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in sets])
    nodes = np.array([v for s in sets for v in sorted(s)], np.int32)
    return off, nodes


def sets_from_csr(off, nodes):
    return [frozenset(int(v) for v in nodes[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


def region_tuple(x: frozenset, y: frozenset, z: frozenset, theta: int = 1):
    """States of the seven Venn regions of (x, y, z), region order (1)..(7)."""
    regs = [x - y - z, y - z - x, z - x - y, (x & y) - z, (y & z) - x, (z & x) - y, x & y & z]
    return tuple(0 if len(r) == 0 else (1 if len(r) <= theta else 2) for r in regs)


def canonical_of_sets(x, y, z, theta: int = 1):
    """Smallest region tuple over the six orders of the actual hyperedges."""
    return min(region_tuple(*p, theta=theta) for p in itertools.permutations((x, y, z)))


def connected(x, y, z) -> bool:
    return sum(bool(p & q) for p, q in ((x, y), (y, z), (z, x))) >= 2


def brute_force_py(sets, theta: int = 1):
    """{canonical ternary tuple: count} over all connected triples."""
    out: dict = {}
    for x, y, z in itertools.combinations(sets, 3):
        if connected(x, y, z):
            c = canonical_of_sets(x, y, z, theta)
            out[c] = out.get(c, 0) + 1
    return out


def brute_force_c(sets, n_nodes: int):
    """Same as brute_force_py, in C, for graphs with millions of triples."""
    os.makedirs(os.path.dirname(_BF_BIN), exist_ok=True)
    if not os.path.exists(_BF_BIN) or os.path.getmtime(_BF_BIN) < os.path.getmtime(_BF_SRC):
        tmp = _BF_BIN + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-o", tmp, _BF_SRC])
        os.replace(tmp, _BF_BIN)
    lines = [f"{n_nodes} {len(sets)}"]
    lines += [" ".join([str(len(s))] + [str(v) for v in sorted(s)]) for s in sets]
    res = subprocess.run([_BF_BIN], input="\n".join(lines) + "\n", capture_output=True,
                         text=True, check=True)
    out = {}
    for line in res.stdout.split("\n"):
        if line.strip():
            t, c = line.split()
            out[tuple(int(ch) for ch in t)] = int(c)
    return out


def counts_by_tuple(t_pattern, counts_3h):
    """Map 3h counts (index id-1) to {canonical tuple: count}, dropping zeros."""
    return {tuple(int(v) for v in t_pattern[i]): int(c)
            for i, c in enumerate(counts_3h) if c}


def micro_graph(seed: int, n_nodes: int = 12, n_edges: int = 30, s_max: int = 6):
    """A small random hypergraph with distinct hyperedges (pure numpy)."""
    rng = np.random.default_rng(seed)
    sets, seen = [], set()
    while len(sets) < n_edges:
        s = frozenset(rng.choice(n_nodes, size=int(rng.integers(1, s_max + 1)),
                                 replace=False).tolist())
        if s not in seen:
            seen.add(s)
            sets.append(s)
    return sets


def realise(pattern):
    """Three hyperedges with 1 node per state-1 region, 2 per state-2 region."""
    roles = [{0}, {1}, {2}, {0, 1}, {1, 2}, {2, 0}, {0, 1, 2}]
    sets = [set(), set(), set()]
    nxt = 0
    for r, st in enumerate(pattern):
        for _ in range(int(st)):
            for who in roles[r]:
                sets[who].add(nxt)
            nxt += 1
    return [frozenset(s) for s in sets], nxt


def canonical_tuple(p):
    """Smallest region tuple over the six relabellings of the three
    hyperedges of a pattern given as states of regions (1)..(7)."""
    member = [1, 2, 4, 3, 6, 5, 7]
    region = {m: r for r, m in enumerate(member)}
    best = None
    for perm in itertools.permutations(range(3)):
        q = [0] * 7
        for r, m in enumerate(member):
            m2 = sum(1 << perm[b] for b in range(3) if m & (1 << b))
            q[region[m2]] = p[r]
        q = tuple(q)
        best = q if best is None or q < best else best
    return best
