"""Star node profiles (mochy_star_node_profile) on the GPU against the oracle.

Every row (the instances of each h-motif and 3h-motif among the hyperedges
that contain one node) must equal the oracle's as int64, on uniform, Zipf,
wide (hyperedges above 32 nodes) and small random hypergraphs and for theta
1 and 2; row v must sum to C(|E_v|, 3).
"""
from math import comb

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
        sets = _util.micro_graph(710 + s, n_nodes=12 + s, n_edges=25 + 3 * s, s_max=6)
        out.append((12 + s, *_util.csr_from_sets(sets)))
    sets = _util.micro_graph(810, n_nodes=70, n_edges=30, s_max=50)
    out.append((70, *_util.csr_from_sets(sets)))
    return out


@pytest.mark.parametrize("theta", [1, 2])
def test_profiles_match_oracle(theta):
    for gi, (n, off, nodes) in enumerate(_graphs()):
        with B.Context(theta=theta) as c:
            c.load(n, off, nodes)
            c.project()
            np_h, np_3h = c.star_node_profile()
            _, doff, dnodes = c.hypergraph()
        o_h, o_3h = oracle.star_node_profile(n, off, nodes, theta=theta)
        assert np.array_equal(np_3h, o_3h), gi
        assert np.array_equal(np_h, o_h), gi
        deg = np.bincount(dnodes, minlength=n)
        assert np.array_equal(np_h.sum(axis=1), [comb(int(d), 3) for d in deg]), gi


def test_needs_projection():
    with B.Context() as c:
        c.load(synth.TINY.n_nodes, *synth.generate(synth.TINY))
        with pytest.raises(B.MochyError) as e:
            B.mochy_star_node_profile(c.h, synth.TINY.n_nodes)
        assert e.value.code == B.E_NOT_PROJECTED
