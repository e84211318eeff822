"""Pins of the oracle's sampling estimators, MoCHy-A and MoCHy-A+ (CPU only).

* Philox4x32-10 against the published known-answer vectors of its authors'
  Random123 distribution (Salmon et al., SC'11).
* The sampling bodies run once per anchor must give 3 M[t] (MoCHy-A, proof of
  Theorem 2, Eq. "Xij:exp") and w[t] M[t] (MoCHy-A+, Eq. "wt", "Yij:exp").
* Unbiasedness over seeds (Theorems 2 and 5).
"""
import numpy as np
import pytest

import oracle
from tests import _util


def test_philox_known_answers():
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
        ([0xffffffff] * 4, [0xffffffff] * 2, [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
        ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
         [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]),
    ]
    for ctr, key, want in kat:
        assert list(oracle.philox(ctr, key)) == want


@pytest.fixture(scope="module")
def T():
    return oracle.tables()


@pytest.mark.parametrize("seed", range(6))
def test_all_anchor_identities(T, seed):
    sets = _util.micro_graph(300 + seed, n_nodes=12, n_edges=40, s_max=5)
    off, nodes = _util.csr_from_sets(sets)
    h, h3 = oracle.count_exact(off, nodes)
    ah, a3 = oracle.count_all_anchors(off, nodes, oracle.A)
    assert np.array_equal(ah, 3 * h) and np.array_equal(a3, 3 * h3)
    ph, p3 = oracle.count_all_anchors(off, nodes, oracle.A_PLUS)
    w_h = np.where(T["h_open"] == 1, 2, 3)
    assert np.array_equal(ph, w_h * h)
    assert np.array_equal(p3, w_h[T["t_to_h"] - 1] * h3)


def test_unbiased_over_seeds(T):
    sets = _util.micro_graph(77, n_nodes=12, n_edges=36, s_max=5)
    off, nodes = _util.csr_from_sets(sets)
    h, _ = oracle.count_exact(off, nodes)
    n_w, _, _ = oracle.project(off, nodes)
    for method, samples in ((oracle.A, 6), (oracle.A_PLUS, 25)):
        est = np.array([oracle.count_sampled(off, nodes, method, samples, seed)[2]
                        for seed in range(300)])
        mean, se = est.mean(0), est.std(0, ddof=1) / np.sqrt(len(est))
        for t in range(26):
            if h[t] > 0:
                assert abs(mean[t] - h[t]) <= 4.5 * se[t] + 1e-9, (method, t)
            else:
                assert np.all(est[:, t] == 0)


def test_estimate_scaling(T):
    sets = _util.micro_graph(78, n_nodes=12, n_edges=36, s_max=5)
    off, nodes = _util.csr_from_sets(sets)
    n_w, _, _ = oracle.project(off, nodes)
    rh, r3, eh, e3 = oracle.count_sampled(off, nodes, oracle.A_PLUS, 50, 9)
    w_h = np.where(T["h_open"] == 1, 2.0, 3.0)
    assert np.array_equal(eh, rh.astype(np.float64) * float(n_w) / (w_h * 50.0))
    rh, r3, eh, e3 = oracle.count_sampled(off, nodes, oracle.A, 20, 9)
    assert np.array_equal(eh, rh.astype(np.float64) * float(len(sets)) / (3.0 * 20.0))
    # raw 3h counts merge into raw h counts
    merged = np.zeros(26, np.int64)
    np.add.at(merged, T["t_to_h"] - 1, r3)
    assert np.array_equal(merged, rh)


def test_same_seed_same_sample():
    sets = _util.micro_graph(79)
    off, nodes = _util.csr_from_sets(sets)
    a = oracle.count_sampled(off, nodes, oracle.A_PLUS, 40, 123)
    b = oracle.count_sampled(off, nodes, oracle.A_PLUS, 40, 123)
    c = oracle.count_sampled(off, nodes, oracle.A_PLUS, 40, 124)
    assert np.array_equal(a[1], b[1]) and not np.array_equal(a[1], c[1])
