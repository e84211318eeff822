"""Pins of the oracle's null model and profile (CPU only).

* Chung-Lu (Algorithm "randomized_hypergraph_alg") draws |E'| (node, hyperedge)
  pairs with P(v) = d_v / |E'| and P(e_j) = |e_j| / |E'|; after the set
  transform (Algorithm "transform") a node v lies in hyperedge j with
  probability 1 - (1 - p_v q_j)^|E'|.  Mean node degrees and the mean total
  size over many copies are checked against that closed form.
* Significance and CP (Eq. "significance", Eq. "cp"): ||CP|| = 1,
  |CP_t| <= 1, recomputation from the returned counts, and the all-zero case.
"""
import numpy as np

import oracle
from tests import _util


def _expected_degrees(sets, n_nodes):
    total = sum(len(s) for s in sets)
    d = np.zeros(n_nodes)
    for s in sets:
        for v in s:
            d[v] += 1
    p = d / total
    q = np.array([len(s) for s in sets]) / total
    inc = 1.0 - (1.0 - np.outer(p, q)) ** total
    return inc.sum(1), inc.sum()


def test_chung_lu_closed_form():
    rng = np.random.default_rng(11)
    n_nodes = 60
    sets = []
    while len(sets) < 25:
        s = frozenset(rng.choice(n_nodes, size=int(rng.integers(6, 10)), replace=False).tolist())
        if s not in sets:
            sets.append(s)
    off, nodes = _util.csr_from_sets(sets)
    exp_deg, exp_total = _expected_degrees(sets, n_nodes)
    n_copies = 400
    degs = np.zeros((n_copies, n_nodes))
    totals = np.zeros(n_copies)
    for c in range(n_copies):
        o2, n2 = oracle.randomize(n_nodes, off, nodes, seed=5, copy=c)
        assert np.all(np.diff(o2) > 0)                     # no empty hyperedge
        rs = _util.sets_from_csr(o2, n2)
        assert len(set(rs)) == len(rs)                      # no duplicate
        degs[c] = np.bincount(n2, minlength=n_nodes)
        totals[c] = n2.size
    se = degs.std(0, ddof=1) / np.sqrt(n_copies) + 1e-12
    z = (degs.mean(0) - exp_deg) / se
    assert np.all(np.abs(z[exp_deg > 0]) < 5.0)
    assert np.all(degs[:, exp_deg == 0] == 0)
    zt = (totals.mean() - exp_total) / (totals.std(ddof=1) / np.sqrt(n_copies))
    assert abs(zt) < 5.0


def test_copies_are_seeded():
    sets = _util.micro_graph(3, n_nodes=20, n_edges=30)
    off, nodes = _util.csr_from_sets(sets)
    a = oracle.randomize(20, off, nodes, 7, 0)
    b = oracle.randomize(20, off, nodes, 7, 0)
    c = oracle.randomize(20, off, nodes, 7, 1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not (np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]))


def test_profile_formula_and_norm():
    sets = _util.micro_graph(21, n_nodes=14, n_edges=40, s_max=5)
    off, nodes = _util.csr_from_sets(sets)
    R = 4
    P = oracle.profile(14, off, nodes, n_random=R, seed=3)
    h, h3 = oracle.count_exact(off, nodes)
    assert np.array_equal(P["counts_h"][0], h) and np.array_equal(P["counts_3h"][0], h3)
    for c in range(R):
        o2, n2 = oracle.randomize(14, off, nodes, 3, c)
        ch, c3 = oracle.count_exact(o2, n2)
        assert np.array_equal(P["counts_h"][1 + c], ch)
        assert np.array_equal(P["counts_3h"][1 + c], c3)
    for key, cnt in (("h", P["counts_h"]), ("3h", P["counts_3h"])):
        m = cnt[0].astype(np.float64)
        mr = cnt[1:].sum(0) / R
        sig = (m - mr) / (m + mr + 1.0)
        assert np.allclose(P["sig_" + key], sig, rtol=1e-15, atol=0)
        cp = P["cp_" + key]
        assert abs(np.linalg.norm(cp) - 1.0) < 1e-12 and np.all(np.abs(cp) <= 1.0)
        assert np.allclose(cp, sig / np.linalg.norm(sig), rtol=1e-14, atol=1e-300)
    assert list(P["degenerate"]) == [0, 0]


def test_profile_degenerate():
    off, nodes = _util.csr_from_sets([frozenset({0, 1})])
    P = oracle.profile(2, off, nodes, n_random=3, seed=1)
    assert np.all(P["sig_h"] == 0) and np.all(P["cp_h"] == 0)
    assert list(P["degenerate"]) == [1, 1]
