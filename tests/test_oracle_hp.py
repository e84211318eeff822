"""Pins of the oracle's hyperedge profiles (Section 3.1, "Hyperedge Profile
(HP)": the t-th element of HP(e) is the number of instances of motif t that
include e).

Checked against brute force over every triple of small random hypergraphs
(each connected triple adds one to the rows of its three hyperedges), and
by the identity that every instance includes exactly three hyperedges:
summed over hyperedges, the profiles are three times the motif counts.
"""
import itertools

import numpy as np

import oracle
from tests import _util


def _brute_hp(sets, theta=1):
    rows = [dict() for _ in sets]
    for (i, x), (j, y), (k, z) in itertools.combinations(list(enumerate(sets)), 3):
        if _util.connected(x, y, z):
            c = _util.canonical_of_sets(x, y, z, theta)
            for e in (i, j, k):
                rows[e][c] = rows[e].get(c, 0) + 1
    return rows


def test_profiles_match_brute_force_on_micro_graphs():
    T = oracle.tables()
    for seed in range(8):
        sets = _util.micro_graph(900 + seed, n_nodes=10 + seed, n_edges=18 + 2 * seed, s_max=5)
        off, nodes = _util.csr_from_sets(sets)
        for theta in (1, 2):
            hp_h, hp_3h = oracle.hyperedge_profile(off, nodes, theta=theta)
            brute = _brute_hp(sets, theta)
            assert hp_3h.shape == (len(sets), 431)
            for e in range(len(sets)):
                assert _util.counts_by_tuple(T["t_pattern"], hp_3h[e]) == brute[e], (seed, e)


def test_profiles_sum_to_three_times_the_counts():
    sets = _util.micro_graph(77, n_nodes=30, n_edges=60, s_max=8)
    off, nodes = _util.csr_from_sets(sets)
    hp_h, hp_3h = oracle.hyperedge_profile(off, nodes)
    h, h3 = oracle.count_exact(off, nodes)
    assert np.array_equal(hp_h.sum(axis=0), 3 * h)
    assert np.array_equal(hp_3h.sum(axis=0), 3 * h3)
    # every h-motif row is the sum of its 3h-motif subdivisions
    t2h = oracle.tables()["t_to_h"]
    folded = np.zeros_like(hp_h)
    for t in range(431):
        folded[:, int(t2h[t]) - 1] += hp_3h[:, t]
    assert np.array_equal(folded, hp_h)


def test_isolated_hyperedge_has_an_empty_profile():
    sets = [frozenset({0, 1}), frozenset({1, 2}), frozenset({2, 3}), frozenset({7, 8})]
    off, nodes = _util.csr_from_sets(sets)
    hp_h, _ = oracle.hyperedge_profile(off, nodes)
    # one connected triple (an open chain); {7, 8} meets nothing
    assert hp_h[3].sum() == 0 and hp_h[:3].sum() == 3 and (hp_h[:3].sum(axis=1) == 1).all()
