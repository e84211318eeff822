"""Pins of the oracle's extensions (CPU only): kh-motifs (Section 4.1
"Extensions Beyond Ternary"), radial node profiles (Section 3.1 "Node
Profile (NP)"), instance enumeration (Algorithm "alg:enum") and the
significance / characteristic profile (Eq. "significance", Eq. "cp").

Each is checked against something other than itself: the motif counts X(k)
printed in the paper, brute force over the triples of micro graphs written
from the definitions, hand-computed fractions, and the relations that must
hold between the variants (merging states, ego-network inclusion).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2310_15668_gb300 import synth
from tests import _util


def _k_states(sets_xyz, k, thr):
    """States of the seven regions of three node sets, k states with the
    k - 2 ascending thresholds thr (0 when empty, else 1 + #exceeded)."""
    x, y, z = sets_xyz
    regs = [x - y - z, y - z - x, z - x - y, (x & y) - z, (y & z) - x, (z & x) - y, x & y & z]
    out = []
    for r in regs:
        c = len(r)
        out.append(0 if c == 0 else 1 + sum(c > t for t in thr))
    return tuple(out)


def _brute_kh(sets, k, thr):
    """{canonical k-state tuple: count} over all connected triples."""
    res = {}
    for x, y, z in itertools.combinations(sets, 3):
        if not _util.connected(x, y, z):
            continue
        c = min(_k_states(p, k, thr) for p in itertools.permutations((x, y, z)))
        res[c] = res.get(c, 0) + 1
    return res


def test_kh_table_sizes_are_the_papers():
    """X(k) = k(k-1)(k^5 + k^4 + 4k^3 + k^2 - 4k + 2)/6: 26, 431, 3,076,
    14,190 for k = 2..5 (Appendix "Number of kH-motifs")."""
    for k, want in ((2, 26), (3, 431), (4, 3076), (5, 14190)):
        assert oracle.kh_tables(k)["to_h"].size == want
        assert k * (k - 1) * (k ** 5 + k ** 4 + 4 * k ** 3 + k ** 2 - 4 * k + 2) // 6 == want


def test_kh_tables_refine_the_h_motifs():
    """Every kh-motif refines one h-motif (its pattern with states > 0 read
    as non-empty), the k = 3 tables are the 3h-motif tables, and h-motif 1
    splits into k(k-1)^2/2 kh-motifs (Appendix "Number of kH-motifs")."""
    T = oracle.tables()
    for k in (3, 4):
        K = oracle.kh_tables(k)
        for i in range(K["to_h"].size):
            b = _canon(tuple(int(v > 0) for v in K["pattern"][i]))
            assert tuple(int(v) for v in T["h_pattern"][K["to_h"][i] - 1]) == b
        assert int((K["to_h"] == 1).sum()) == k * (k - 1) ** 2 // 2
    K3 = oracle.kh_tables(3)
    assert np.array_equal(K3["pattern"], T["t_pattern"])
    assert np.array_equal(K3["to_h"], T["t_to_h"])


@pytest.mark.parametrize("seed", range(8))
def test_4h_counts_match_brute_force(seed):
    sets = _util.micro_graph(900 + seed, n_nodes=14, n_edges=24, s_max=9)
    off, nodes = _util.csr_from_sets(sets)
    thr = (1, 2) if seed % 2 == 0 else (2, 4)
    h, kh = oracle.count_exact_kh(off, nodes, 4, thr)
    K = oracle.kh_tables(4)
    got = {tuple(int(v) for v in K["pattern"][i]): int(c) for i, c in enumerate(kh) if c}
    assert got == _brute_kh(sets, 4, thr)
    assert np.array_equal(h, oracle.count_exact(off, nodes)[0])


def test_4h_counts_merge_into_3h_counts():
    """With thresholds (1, 2), merging states 2 and 3 gives the 3h-motifs of
    theta = 1 and merging states 1 and 2 those of theta = 2."""
    spec = synth.HypergraphSpec(300, 600, 2, 12, "powerlaw", 2.0, "zipf", 0.9, seed=4)
    off, nodes = synth.generate(spec)
    _, kh = oracle.count_exact_kh(off, nodes, 4, (1, 2))
    K = oracle.kh_tables(4)
    for theta, merge in ((1, {0: 0, 1: 1, 2: 2, 3: 2}), (2, {0: 0, 1: 1, 2: 1, 3: 2})):
        T = oracle.tables()
        _, h3 = oracle.count_exact(off, nodes, theta=theta)
        want = _util.counts_by_tuple(T["t_pattern"], h3)
        got = {}
        for i, c in enumerate(kh):
            if not c:
                continue
            # merging states can change which permutation is smallest
            sets_pat = tuple(merge[int(v)] for v in K["pattern"][i])
            key = _canon(sets_pat)
            got[key] = got.get(key, 0) + int(c)
        assert got == want


_canon = _util.canonical_tuple


def _radial_brute(sets, n_nodes):
    out = []
    for v in range(n_nodes):
        ev = [s for s in sets if v in s]
        vv = frozenset().union(*ev) if ev else frozenset()
        rv = [s for s in sets if s <= vv] if ev else []
        out.append(_util.brute_force_py(rv))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_radial_profiles_match_brute_force(seed):
    n = 12
    sets = _util.micro_graph(950 + seed, n_nodes=n, n_edges=20, s_max=5)
    off, nodes = _util.csr_from_sets(sets)
    T = oracle.tables()
    _, r3 = oracle.radial_node_profile(n, off, nodes)
    want = _radial_brute(sets, n)
    for v in range(n):
        assert _util.counts_by_tuple(T["t_pattern"], r3[v]) == want[v]


def test_radial_contains_star():
    """E_v is a subset of R_v, so every star instance is a radial instance;
    when every hyperedge holds v, R_v = E and the profile is the full count."""
    spec = synth.HypergraphSpec(60, 120, 2, 6, "uniform", 0.0, "zipf", 1.0, seed=6)
    off, nodes = synth.generate(spec)
    _, s3 = oracle.star_node_profile(60, off, nodes)
    _, r3 = oracle.radial_node_profile(60, off, nodes)
    assert (r3 >= s3).all()
    star = [frozenset({0} | s) for s in _util.micro_graph(3, n_nodes=9, n_edges=15, s_max=4)]
    star = list(dict.fromkeys(star))
    off2, nodes2 = _util.csr_from_sets(star)
    rh, r32 = oracle.radial_node_profile(9, off2, nodes2)
    fh, f3 = oracle.count_exact(off2, nodes2)
    assert np.array_equal(rh[0], fh) and np.array_equal(r32[0], f3)


@pytest.mark.parametrize("seed", range(4))
def test_enumeration_lists_every_connected_triple_once(seed):
    sets = _util.micro_graph(980 + seed, n_nodes=12, n_edges=22, s_max=5)
    off, nodes = _util.csr_from_sets(sets)
    T = oracle.tables()
    rows, n = oracle.enumerate_instances(off, nodes)
    assert n == rows.shape[0]
    want = {}
    for i, j, k in itertools.combinations(range(len(sets)), 3):
        x, y, z = sets[i], sets[j], sets[k]
        if _util.connected(x, y, z):
            want[(i, j, k)] = _util.canonical_of_sets(x, y, z)
    got = {}
    for i, j, k, h, h3 in rows.tolist():
        assert (i, j, k) not in got                         # written once
        got[(i, j, k)] = tuple(int(v) for v in T["t_pattern"][h3 - 1])
        assert T["t_to_h"][h3 - 1] == h
    assert got == want
    h_all, _ = oracle.count_exact(off, nodes)
    assert n == int(h_all.sum())


def test_enumeration_cap():
    off, nodes = synth.generate(synth.TINY)
    rows, n = oracle.enumerate_instances(off, nodes, cap=100)
    assert rows.shape == (100, 5) and n == int(oracle.count_exact(off, nodes)[0].sum())


def test_significance_and_cp_by_hand():
    """Eq. "significance" with eps = 1 and M_rand the mean of two copies:
    M = (10, 0, 5, 3), copy sums (8, 4, 10, 0) -> M_rand = (4, 2, 5, 0),
    Delta = (6/15, -2/3, 0, 3/4) = (2/5, -2/3, 0, 3/4); ||Delta||^2 =
    4/25 + 4/9 + 9/16 = 4201/3600, so CP = (24, -40, 0, 45) / sqrt(4201)."""
    sig, cp, deg = oracle.significance_cp([10, 0, 5, 3], [8, 4, 10, 0], 2, eps=1.0)
    assert not deg
    np.testing.assert_allclose(sig, [2 / 5, -2 / 3, 0.0, 3 / 4], rtol=1e-15, atol=0)
    r = math.sqrt(4201.0)
    np.testing.assert_allclose(cp, [24 / r, -40 / r, 0.0, 45 / r], rtol=1e-14, atol=0)
    # eps enters the denominator only: eps = 3 gives (6/17, -2/5, 0, 3/6)
    sig3, _, _ = oracle.significance_cp([10, 0, 5, 3], [8, 4, 10, 0], 2, eps=3.0)
    np.testing.assert_allclose(sig3, [6 / 17, -2 / 5, 0.0, 1 / 2], rtol=1e-15, atol=0)


def test_copies_equal_to_the_input_give_zero_significance():
    """If every randomized copy had the input's counts, M_rand = M and every
    significance is 0; the CP is then 0/0, returned as zeros with the
    degenerate flag (reading R9)."""
    M = np.array([7, 0, 123456789, 2, 1], np.int64)
    sig, cp, deg = oracle.significance_cp(M, 5 * M, 5)
    assert deg and not sig.any() and not cp.any()
