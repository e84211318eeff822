"""The sampling estimators of the oracle against the paper's bias-and-variance
theorems (Theorem "Bias and Variance of MoCHy-A": Eq. "sampling_ver1:
variance"; Theorem "Bias and Variance of MoCHy-A+": Eqs. "sampling_ver2:
variance:closed" / ":open").

A one-draw estimate must equal, exactly, the contribution of the drawn
anchor: for MoCHy-A the number of instances of each h-motif that contain
the drawn hyperedge, for MoCHy-A+ the number that contain the drawn
hyperwedge (brute force over all triples).  The exact variance over all
anchors must then equal the theorems' expressions, in rational arithmetic,
with p_l[t] (q_n[t]) read as the number of ORDERED pairs of distinct
instances of motif t that share l hyperedges (n hyperwedges): the text's
"pairs" is ambiguous, and only the ordered reading makes the stated
formulas the variance of the stated estimators; the unordered reading is
checked to fail.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import _util


def _draw(seed, stream, rng):
    # draw 0 of stream `stream`: Philox4x32-10 counter (0, 0, stream, 0), key
    # (seed_lo, seed_hi); the 64-bit output u selects floor(u * rng / 2^64)
    o = oracle.philox([0, 0, stream, 0], [seed & 0xFFFFFFFF, seed >> 32])
    u = (int(o[1]) << 32) | int(o[0])
    return (u * rng) >> 64


def _instances(sets, T):
    by_tuple = {tuple(int(v) for v in T["t_pattern"][i]): i for i in range(431)}
    out = []
    for i, j, k in itertools.combinations(range(len(sets)), 3):
        x, y, z = sets[i], sets[j], sets[k]
        if _util.connected(x, y, z):
            t3 = by_tuple[_util.canonical_of_sets(x, y, z)]
            out.append(((i, j, k), int(T["t_to_h"][t3])))
    return out


def _wedges_of(inst, sets):
    i, j, k = inst
    return {(p, q) for p, q in ((i, j), (i, k), (j, k)) if sets[p] & sets[q]}


@pytest.fixture(scope="module")
def case():
    T = oracle.tables()
    sets = _util.micro_graph(4242, n_nodes=11, n_edges=26, s_max=4)
    off, nodes = _util.csr_from_sets(sets)
    inst = _instances(sets, T)
    wedges = sorted((p, q) for p, q in itertools.combinations(range(len(sets)), 2)
                    if sets[p] & sets[q])
    X = np.zeros((len(sets), 26), np.int64)          # per hyperedge (MoCHy-A anchor)
    Y = {w: np.zeros(26, np.int64) for w in wedges}  # per hyperwedge (MoCHy-A+ anchor)
    for members, h in inst:
        for e in members:
            X[e, h - 1] += 1
        for w in _wedges_of(members, sets):
            Y[w][h - 1] += 1
    return dict(T=T, sets=sets, off=off, nodes=nodes, inst=inst, wedges=wedges, X=X, Y=Y)


def test_one_draw_equals_the_anchor_contribution(case):
    E, W = len(case["sets"]), len(case["wedges"])
    for seed in range(60):
        raw_a = oracle.count_sampled(case["off"], case["nodes"], oracle.A, 1, seed)[0]
        assert np.array_equal(raw_a, case["X"][_draw(seed, 1, E)]), seed
        raw_p = oracle.count_sampled(case["off"], case["nodes"], oracle.A_PLUS, 1, seed)[0]
        assert np.array_equal(raw_p, case["Y"][case["wedges"][_draw(seed, 2, W)]]), seed


def _pairs(inst, t, shared):
    """counts[l] = ordered pairs of distinct instances of motif t sharing l items"""
    items = [shared(m) for m, h in inst if h == t]
    counts = {}
    for a in range(len(items)):
        for b in range(len(items)):
            if a != b:
                lvl = len(items[a] & items[b])
                counts[lvl] = counts.get(lvl, 0) + 1
    return counts


def _var(values, scale):
    # variance of scale * (value of one uniformly drawn anchor)
    n = len(values)
    m1 = Fraction(sum(values), n)
    m2 = Fraction(sum(v * v for v in values), n)
    return scale * scale * (m2 - m1 * m1)


def test_variance_theorems(case):
    sets, inst, T = case["sets"], case["inst"], case["T"]
    E, W = len(sets), len(case["wedges"])
    h_open = T["h_open"]
    checked_unordered_fails = False
    for t in range(1, 27):
        M = sum(1 for _, h in inst if h == t)
        if M == 0:
            continue
        # MoCHy-A, one sample: scale |E| / 3
        p = _pairs(inst, t, lambda m: set(m))
        direct = _var([int(case["X"][e, t - 1]) for e in range(E)], Fraction(E, 3))
        paper = Fraction(1, 3) * M * (E - 3) + Fraction(1, 9) * sum(
            p.get(l, 0) * (l * E - 9) for l in range(3))
        assert direct == paper, ("A", t)
        unordered = Fraction(1, 3) * M * (E - 3) + Fraction(1, 9) * sum(
            Fraction(p.get(l, 0), 2) * (l * E - 9) for l in range(3))
        if p.get(1, 0) + p.get(2, 0) > 0 and unordered != direct:
            checked_unordered_fails = True
        # MoCHy-A+, one sample: scale |wedges| / w[t], w = 2 open, 3 closed
        w = 2 if h_open[t - 1] else 3
        q = _pairs(inst, t, lambda m: _wedges_of(m, sets))
        direct = _var([int(case["Y"][wd][t - 1]) for wd in case["wedges"]], Fraction(W, w))
        paper = Fraction(1, w) * M * (W - w) + Fraction(1, w * w) * sum(
            q.get(n, 0) * (n * W - w * w) for n in range(2))
        assert direct == paper, ("A+", t)
        assert set(q) <= {0, 1}                     # two instances share at most one hyperwedge
    assert checked_unordered_fails
