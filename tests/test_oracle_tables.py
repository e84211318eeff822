"""Pins of the oracle's motif tables (CPU only).

Pinned against numbers the paper prints and against the definition by
isomorphism (Section 2.2 "Equivalently, when we leave at most one node in each
of the above subsets ..."; Section 4.1 the same with min(ceil(c/theta), 2)
nodes).
"""
import itertools

import numpy as np
import pytest

import oracle
from tests import _util


@pytest.fixture(scope="module")
def T():
    return oracle.tables()


def test_filter_chain_matches_paper(T):
    # Table "hmotif_cnt_table", 3-hyperedge column: 128 -> 40 -> 30 -> 26.
    assert list(T["chain"][:4]) == [128, 40, 30, 26]
    # Section 4.1: "Out of the 3^7 possible patterns, 431 3h-motifs remain".
    assert T["chain"][4] == 2187 and T["chain"][7] == 431


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_kh_motif_count_formula(k):
    # Eq. "kh_motif_cnt": X(k) = k(k-1)(k^5+k^4+4k^3+k^2-4k+2)/6; Section 4.1
    # prints 3,076 for k = 4.
    x = k * (k - 1) * (k ** 5 + k ** 4 + 4 * k ** 3 + k ** 2 - 4 * k + 2) // 6
    assert oracle.count_kh(k) == x
    if k == 4:
        assert x == 3076


def test_open_ids_are_17_to_22(T):
    # Fig. "motif_three_hyperedges": h-motifs 17-22 are open.
    assert list(np.nonzero(T["h_open"])[0] + 1) == [17, 18, 19, 20, 21, 22]


def test_h16_has_all_regions(T):
    # Section 5.2: in h-motif 16 all seven regions are non-empty.
    assert list(T["h_pattern"][15]) == [1] * 7
    assert sum(1 for p in T["h_pattern"] if all(p)) == 1


def test_h17_h18_are_hyperedge_with_two_disjoint_subsets(T):
    # Section 5.2: instances of 17 and 18 consist of a hyperedge and two
    # disjoint subsets of it.
    for hid in (17, 18):
        sets, _ = _util.realise(T["h_pattern"][hid - 1])
        big = max(sets, key=len)
        small = [s for s in sets if s is not big]
        assert all(s < big for s in small) and not (small[0] & small[1])


def test_subdivisions(T):
    # Section 4.1 / Appendix "Number of kH-motifs": h-motif 1 splits into six
    # 3h-motifs, which are 3h-motifs 1-6; all subdivisions sum to 431.
    t2h = T["t_to_h"]
    assert list(t2h[:6]) == [1] * 6 and t2h[6] != 1
    assert np.all(np.diff(t2h) >= 0)
    assert sorted(set(t2h.tolist())) == list(range(1, 27))
    # per h-motif with n non-empty regions split into orbits, the count of
    # subdivisions equals the number of orbit-respecting 2-colourings
    assert len(t2h) == 431


def test_luts_agree_with_isomorphism_definition(T):
    """Each table id, realised as sets, is recognised by set canonicalisation."""
    tp, hp = T["t_pattern"], T["h_pattern"]
    for tid in range(1, 432):
        sets, _ = _util.realise(tp[tid - 1])
        assert len(set(sets)) == 3 and _util.connected(*sets)
        assert _util.canonical_of_sets(*sets) == tuple(int(v) for v in tp[tid - 1])
        b = tuple(1 if v else 0 for v in tp[tid - 1])
        hid = T["t_to_h"][tid - 1]
        bsets, _ = _util.realise(b)
        assert _util.canonical_of_sets(*bsets, theta=10 ** 6) == \
            tuple(int(v) for v in hp[hid - 1])


def test_lut_covers_every_code(T):
    """A code maps to id 0 exactly when its realisation is invalid."""
    for code in range(2187):
        digits, x = [], code
        for _ in range(7):
            digits.append(x % 3)
            x //= 3
        sets, _ = _util.realise(digits)
        valid = len(set(sets)) == 3 and _util.connected(*sets)
        tid = T["lut_3h"][code]
        assert (tid != 0) == valid
        if valid:
            assert tuple(int(v) for v in T["t_pattern"][tid - 1]) == \
                _util.canonical_of_sets(*sets)
            bcode = sum((1 if d else 0) << p for p, d in enumerate(digits))
            assert T["lut_h"][bcode] == T["t_to_h"][tid - 1]


def _pairwise_classes(T, full: bool):
    def key_of(sets):
        best = None
        for p in itertools.permutations(sets):
            if full:
                key = tuple((bool(a & b), bool(a - b), bool(b - a))
                            for a, b in itertools.combinations(p, 2))
            else:
                key = tuple(bool(a & b) for a, b in itertools.combinations(p, 2))
            best = key if best is None or key < best else best
        return best
    keys = {}
    for hid in range(1, 27):
        sets, _ = _util.realise(T["h_pattern"][hid - 1])
        keys.setdefault(key_of(sets), []).append(hid)
    return list(keys.values())


def test_pairwise_overlaps_give_eight_patterns_and_twelve_shared(T):
    """Section 2.2 "Why multi-way overlaps?": pairwise emptiness (e_x & e_y,
    e_x \\ e_y, e_y \\ e_x) allows just eight patterns of three distinct
    hyperedges, 12 of the 26 h-motifs have the same pairwise overlaps, and
    plain adjacency (network motifs) allows two."""
    full = _pairwise_classes(T, True)
    assert len(full) == 8
    assert max(len(c) for c in full) == 12
    assert len(_pairwise_classes(T, False)) == 2
