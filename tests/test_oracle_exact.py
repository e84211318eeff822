"""Pins of the oracle's exact counting, MoCHy-E (CPU only).

Pinned against brute force over all hyperedge triples (an independent
set-based enumeration), pattern-coverage fixtures built from the isomorphism
definition (Section 2.2, Section 4.1), the worked example of Section 2.1 /
Fig. 1, and invariants that hold for any hypergraph.
"""
import numpy as np
import pytest

import oracle
from paper_2310_15668_gb300 import synth
from tests import _util


@pytest.fixture(scope="module")
def T():
    return oracle.tables()


@pytest.mark.parametrize("seed", range(40))
def test_micro_graphs_match_brute_force(T, seed):
    sets = _util.micro_graph(seed, n_nodes=10 + seed % 5, n_edges=18 + seed % 13)
    off, nodes = _util.csr_from_sets(sets)
    h, h3 = oracle.count_exact(off, nodes)
    bf = _util.brute_force_py(sets)
    assert _util.counts_by_tuple(T["t_pattern"], h3) == bf
    # h counts are the 3h counts merged by parent h-motif
    merged = np.zeros(26, np.int64)
    np.add.at(merged, T["t_to_h"] - 1, h3)
    assert np.array_equal(merged, h)


def test_tiny_config_matches_brute_force(T):
    """All C(2000, 3) triples of the tiny workload, enumerated in C."""
    off, nodes = synth.generate(synth.TINY)
    sets = _util.sets_from_csr(off, nodes)
    h, h3 = oracle.count_exact(off, nodes)
    bf = _util.brute_force_c(sets, synth.TINY.n_nodes)
    assert _util.counts_by_tuple(T["t_pattern"], h3) == bf
    assert h.sum() == sum(bf.values()) > 0


def test_every_pattern_counts_once(T):
    """Each of the 431 patterns, realised with 1 node per state-1 region and 2
    per state-2 region plus a disjoint decoy, is one instance of its id."""
    for tid in range(1, 432):
        sets, n = _util.realise(T["t_pattern"][tid - 1])
        decoy = frozenset({n, n + 1})
        off, nodes = _util.csr_from_sets(list(sets) + [decoy])
        h, h3 = oracle.count_exact(off, nodes)
        assert h3.sum() == 1 and h3[tid - 1] == 1
        assert h.sum() == 1 and h[T["t_to_h"][tid - 1] - 1] == 1


def test_worked_example_of_section_2():
    """Section 2.1 / Fig. 1: e_1 = {L, K, F}; the hyperwedges are exactly
    (1,2), (1,3), (2,3), (1,4); {e1,e2,e4} and {e1,e3,e4} have the same
    pairwise overlaps but different h-motifs (Section 2.2).  The node sets of
    e_2..e_4 are lost with the figure; this is one set consistent with every
    stated fact."""
    L, K, F, A, B = 0, 1, 2, 3, 4
    sets = [frozenset({L, K, F}), frozenset({L, K, A}), frozenset({K, B}), frozenset({F})]
    off, nodes = _util.csr_from_sets(sets)
    n_w, _, deg = oracle.project(off, nodes)
    assert n_w == 4 and list(deg) == [3, 2, 2, 1]
    h, _ = oracle.count_exact(off, nodes)
    assert h.sum() == 3                       # {1,2,3}, {1,2,4}, {1,3,4}
    T = oracle.tables()
    closed = [t for t in range(26) if h[t] and not T["h_open"][t]]
    opened = [t for t in range(26) if h[t] and T["h_open"][t]]
    assert len(closed) == 1 and len(opened) == 2   # two different open motifs
    for hid in (x + 1 for x in opened):            # hyperedge + two disjoint subsets?
        assert h[hid - 1] == 1


@pytest.mark.parametrize("seed", range(8))
def test_invariants(T, seed):
    sets = _util.micro_graph(100 + seed, n_nodes=15, n_edges=60, s_max=5)
    off, nodes = _util.csr_from_sets(sets)
    h, h3 = oracle.count_exact(off, nodes)
    n_w, _, deg = oracle.project(off, nodes)
    open_ = sum(h[t] for t in range(26) if T["h_open"][t])
    closed = sum(h[t] for t in range(26) if not T["h_open"][t])
    # every pair of neighbours of e_i is an open triple centred at e_i or a
    # closed one, and a closed triple is seen from each of its three members
    assert open_ + 3 * closed == int((deg * (deg - 1) // 2).sum())
    # |wedges| from degrees
    assert 2 * n_w == int(deg.sum())
    # closed triples are the triangles of the line graph
    adj = [[bool(a & b) and i != j for j, b in enumerate(sets)] for i, a in enumerate(sets)]
    tri = sum(1 for i in range(len(sets)) for j in range(i + 1, len(sets)) if adj[i][j]
              for k in range(j + 1, len(sets)) if adj[i][k] and adj[j][k])
    assert closed == tri


def test_subsets_add_up(T):
    """Per-anchor counts of Algorithm exact_motif_counting add up to the total,
    and the on-the-fly neighbour path equals the projected path."""
    off, nodes = synth.generate(synth.TINY)
    h, h3 = oracle.count_exact(off, nodes)
    e = off.size - 1
    perm = np.random.default_rng(5).permutation(e).astype(np.int32)
    parts = np.array_split(perm, 3)
    acc_h = np.zeros(26, np.int64)
    acc_3h = np.zeros(431, np.int64)
    for p in parts:
        ph, p3 = oracle.count_exact_subset(off, nodes, p)
        acc_h += ph
        acc_3h += p3
    assert np.array_equal(acc_h, h) and np.array_equal(acc_3h, h3)


def test_dedupe_and_sorting():
    sets = [[3, 1, 2], [2, 3, 1], [5], [1, 2, 3, 3], [4, 5], [5]]
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in sets])
    nodes = np.array([v for s in sets for v in s], np.int32)
    o2, n2, dup = oracle.dedupe(off, nodes)
    assert dup == 3
    assert _util.sets_from_csr(o2, n2) == [frozenset({1, 2, 3}), frozenset({5}),
                                           frozenset({4, 5})]
    assert list(n2) == [1, 2, 3, 5, 4, 5]


def test_empty_and_degenerate_graphs():
    # no hyperedge, one hyperedge, two disjoint, two overlapping: no triple
    for sets in ([], [{0}], [{0}, {1}], [{0, 1}, {1, 2}]):
        off, nodes = _util.csr_from_sets([frozenset(s) for s in sets])
        h, h3 = oracle.count_exact(off, nodes)
        assert h.sum() == 0 and h3.sum() == 0
