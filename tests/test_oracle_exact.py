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


def _owned_brute_force(sets, anchor, rank, theta=1):
    """Instances the outer-loop iteration of `anchor` counts under a total
    order `rank` (Algorithm "exact_motif_counting" with i < min(j, k) read as
    rank[i] < min(rank[j], rank[k])): every connected triple that holds the
    anchor and either has it as the centre of an open instance (adjacent to
    both others, which are disjoint) or, when closed, has it lowest-ranked.
    Enumerated from the node sets, {canonical tuple: count}."""
    out = {}
    x = sets[anchor]
    others = [i for i in range(len(sets)) if i != anchor]
    for a in range(len(others)):
        for b in range(a + 1, len(others)):
            j, k = others[a], others[b]
            y, z = sets[j], sets[k]
            if not (x & y and x & z):
                continue                      # the anchor must be adjacent to both
            if y & z and not (rank[anchor] < rank[j] and rank[anchor] < rank[k]):
                continue                      # closed: owned by its lowest-ranked member
            c = _util.canonical_of_sets(x, y, z, theta)
            out[c] = out.get(c, 0) + 1
    return out


@pytest.mark.parametrize("seed", range(6))
def test_ranked_anchor_owns_what_brute_force_says(T, seed):
    """A fixed total order decides which anchor counts a closed instance;
    per anchor the oracle's ranked subset equals the instances enumerated
    from the sets under that order."""
    sets = _util.micro_graph(700 + seed, n_nodes=11, n_edges=22, s_max=5)
    off, nodes = _util.csr_from_sets(sets)
    rank = np.random.default_rng(seed).permutation(len(sets)).astype(np.int64)
    for anchor in range(len(sets)):
        h, h3 = oracle.count_exact_ranked(off, nodes, [anchor], rank)
        assert _util.counts_by_tuple(T["t_pattern"], h3) == _owned_brute_force(sets, anchor, rank)


def test_any_order_counts_every_instance_once():
    """Summed over all anchors, every total order gives the exact count, on
    several host threads as on one."""
    spec = synth.HypergraphSpec(400, 900, 2, 12, "powerlaw", 2.5, "zipf", 0.8, seed=9)
    off, nodes = synth.generate(spec)
    h, h3 = oracle.count_exact(off, nodes)
    e = off.size - 1
    everyone = np.arange(e, dtype=np.int32)
    for seed in range(3):
        rank = np.random.default_rng(seed).permutation(e).astype(np.int64)
        rh, r3 = oracle.count_exact_ranked(off, nodes, everyone, rank, threads=3)
        assert np.array_equal(rh, h) and np.array_equal(r3, h3)
    th, t3 = oracle.count_exact_threads(off, nodes, threads=4)
    assert np.array_equal(th, h) and np.array_equal(t3, h3)
    # with no order given, ids are compared: the plain subset call
    part = everyone[::7]
    assert all(np.array_equal(a, b) for a, b in
               zip(oracle.count_exact_ranked(off, nodes, part),
                   oracle.count_exact_subset(off, nodes, part)))


def test_line_degrees_from_incidence_lists():
    """|N_e| from the incidence lists equals the degree in the projected
    line graph, and Σ_e |N_e| = 2 |wedges|."""
    for spec in (synth.TINY, synth.HypergraphSpec(300, 700, 2, 25, "powerlaw", 2.5, "zipf",
                                                  1.0, seed=2)):
        off, nodes = synth.generate(spec)
        nw, md, deg = oracle.project(off, nodes)
        ld = oracle.line_degrees(off, nodes, threads=3)
        assert np.array_equal(ld, deg)
        assert int(ld.sum()) == 2 * nw and int(ld.max()) == md


def _split_share_brute(sets, r, rank, theta=1):
    """A row's share when open instances are counted per centre from all its
    neighbour pairs: every pair {p, q} of neighbours of r classified as if
    open at r (regions of an open instance from the overlaps with r, when
    they fit in e_r), plus, for a closed instance whose lowest-ranked member
    is r, its pattern minus its as-if-open pattern at each of its three
    centres.  From the node sets, {canonical tuple: count}."""
    def state(c):
        return 0 if c == 0 else (1 if c <= theta else 2)

    def as_if_open(c, p, q):
        C, P, Q = sets[c], sets[p], sets[q]
        wcp, wcq = len(C & P), len(C & Q)
        if wcp + wcq > len(C):
            return None
        regs = (len(C) - wcp - wcq, len(P) - wcp, len(Q) - wcq, wcp, 0, wcq, 0)
        return _util.canonical_tuple(tuple(state(v) for v in regs))

    out = {}

    def add(key, v):
        if key is not None:
            out[key] = out.get(key, 0) + v

    nbrs = [i for i in range(len(sets)) if i != r and sets[i] & sets[r]]
    for a in range(len(nbrs)):
        for b in range(a + 1, len(nbrs)):
            j, k = nbrs[a], nbrs[b]
            add(as_if_open(r, j, k), 1)
            if sets[j] & sets[k] and rank[r] < rank[j] and rank[r] < rank[k]:
                add(_util.canonical_of_sets(sets[r], sets[j], sets[k], theta), 1)
                add(as_if_open(r, j, k), -1)
                add(as_if_open(j, r, k), -1)
                add(as_if_open(k, r, j), -1)
    return {key: v for key, v in out.items() if v}


@pytest.mark.parametrize("seed", range(5))
def test_split_row_shares_match_brute_force(T, seed):
    sets = _util.micro_graph(720 + seed, n_nodes=11, n_edges=22, s_max=5)
    off, nodes = _util.csr_from_sets(sets)
    rank = np.random.default_rng(seed).permutation(len(sets)).astype(np.int64)
    for r in range(len(sets)):
        _, h3 = oracle.count_split_rows(off, nodes, [r], rank)
        assert _util.counts_by_tuple(T["t_pattern"], h3) == _split_share_brute(sets, r, rank)


def test_split_row_shares_sum_to_the_exact_count():
    spec = synth.HypergraphSpec(400, 900, 2, 12, "powerlaw", 2.5, "zipf", 0.8, seed=9)
    off, nodes = synth.generate(spec)
    h, h3 = oracle.count_exact(off, nodes)
    e = off.size - 1
    for seed in range(2):
        rank = np.random.default_rng(seed).permutation(e).astype(np.int64)
        parts = np.array_split(np.random.default_rng(seed + 7).permutation(e).astype(np.int32), 3)
        acc_h = sum(oracle.count_split_rows(off, nodes, p, rank, threads=3)[0] for p in parts)
        acc_3h = sum(oracle.count_split_rows(off, nodes, p, rank, threads=3)[1] for p in parts)
        assert np.array_equal(acc_h, h) and np.array_equal(acc_3h, h3)
