"""Pins of the oracle's star node profiles (Section 3.1, "Node Profile (NP)"
with star ego-networks: the hyperedges that contain v, kept whole).

Checked against brute force over the triples of E_v on small random
hypergraphs; every triple of E_v is an instance (its hyperedges pairwise
share v), so a row sums to C(|E_v|, 3), and every such instance is closed
with a non-empty triple region (h-motifs 1-16 in this numbering).
"""
import itertools
from math import comb

import numpy as np

import oracle
from tests import _util


def test_profiles_match_brute_force_on_micro_graphs():
    T = oracle.tables()
    for seed in range(6):
        n = 10 + seed
        sets = _util.micro_graph(950 + seed, n_nodes=n, n_edges=20 + 2 * seed, s_max=5)
        off, nodes = _util.csr_from_sets(sets)
        for theta in (1, 2):
            np_h, np_3h = oracle.star_node_profile(n, off, nodes, theta=theta)
            assert np_3h.shape == (n, 431)
            for v in range(n):
                ev = [s for s in sets if v in s]
                brute = {}
                for x, y, z in itertools.combinations(ev, 3):
                    c = _util.canonical_of_sets(x, y, z, theta)
                    brute[c] = brute.get(c, 0) + 1
                assert _util.counts_by_tuple(T["t_pattern"], np_3h[v]) == brute, (seed, v)


def test_rows_count_all_triples_of_the_star_and_are_closed():
    n = 40
    sets = _util.micro_graph(61, n_nodes=n, n_edges=80, s_max=7)
    off, nodes = _util.csr_from_sets(sets)
    np_h, np_3h = oracle.star_node_profile(n, off, nodes)
    deg = np.zeros(n, np.int64)
    for s in sets:
        for v in s:
            deg[v] += 1
    assert np.array_equal(np_h.sum(axis=1), [comb(int(d), 3) for d in deg])
    assert np.array_equal(np_3h.sum(axis=1), np_h.sum(axis=1))
    assert np_h[:, 16:].sum() == 0
