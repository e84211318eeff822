"""Hyperedge profiles (mochy_hyperedge_profile) on the GPU against the oracle.

Every row (the instances of each h-motif and 3h-motif that include one
hyperedge) must equal the oracle's as int64, on uniform, Zipf, wide
(hyperedges above 32 nodes) and small random hypergraphs and for theta 1
and 2; summed over hyperedges the profiles must be three times the exact
counts.
"""
import numpy as np
import pytest

import oracle
from paper_2310_15668_gb300 import binding as B, synth
from tests import _util

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _graphs():
    z = synth.HypergraphSpec(500, 1000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=3)
    w = synth.HypergraphSpec(240, 220, 2, 60, "uniform", 0.0, "uniform", 0.0, seed=4)
    out = [(synth.TINY.n_nodes, *synth.generate(synth.TINY)), (z.n_nodes, *synth.generate(z)),
           (w.n_nodes, *synth.generate(w))]
    for s in range(6):
        sets = _util.micro_graph(700 + s, n_nodes=12 + s, n_edges=25 + 3 * s, s_max=6)
        out.append((12 + s, *_util.csr_from_sets(sets)))
    sets = _util.micro_graph(800, n_nodes=70, n_edges=30, s_max=50)
    out.append((70, *_util.csr_from_sets(sets)))
    return out


@pytest.mark.parametrize("theta", [1, 2])
def test_profiles_match_oracle(theta):
    for gi, (n, off, nodes) in enumerate(_graphs()):
        with B.Context(theta=theta) as c:
            c.load(n, off, nodes)
            c.project()
            hp_h, hp_3h = c.hyperedge_profile()
            h, h3 = c.count_exact()
        o_h, o_3h = oracle.hyperedge_profile(off, nodes, theta=theta)
        assert np.array_equal(hp_3h, o_3h), gi
        assert np.array_equal(hp_h, o_h), gi
        assert np.array_equal(hp_h.sum(axis=0), 3 * h), gi
        assert np.array_equal(hp_3h.sum(axis=0), 3 * h3), gi


def test_profiles_sum_to_three_times_the_counts_on_a_larger_graph():
    spec = synth.HypergraphSpec(2500, 5000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=9)
    off, nodes = synth.generate(spec)
    with B.Context() as c:
        c.load(spec.n_nodes, off, nodes)
        c.project()
        hp_h, hp_3h = c.hyperedge_profile()
        h, h3 = c.count_exact()
    assert np.array_equal(hp_h.sum(axis=0), 3 * h)
    assert np.array_equal(hp_3h.sum(axis=0), 3 * h3)
    assert (hp_h >= 0).all()


def test_needs_projection():
    with B.Context() as c:
        c.load(synth.TINY.n_nodes, *synth.generate(synth.TINY))
        with pytest.raises(B.MochyError) as e:
            B.mochy_hyperedge_profile(c.h, 2000)
        assert e.value.code == B.E_NOT_PROJECTED
