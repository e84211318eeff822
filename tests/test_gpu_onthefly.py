"""MoCHy-A+ without the line graph on the GPU (needs a GB300).

mochy_count_sampled_onthefly draws the same hyperwedges as MoCHy-A+ on the
projected line graph and classifies the same instances, so its raw counts
and FP64 estimates must equal the oracle's MoCHy-A+ bit for bit, whatever
share of the nodes gets a membership bitmap (the memoized part) and
whatever the neighbourhood sizes; its |wedges| must equal the oracle's.  On
the medium workload (1.85e9 hyperwedges) it must equal the projected GPU
call on the same draws, and |wedges| the half-sum of the oracle's line
degrees.
"""
import numpy as np
import pytest

import oracle
from paper_2310_15668_gb300 import binding as B, synth
from tests import _util

pytestmark = pytest.mark.gpu

ZIPF_SMALL = synth.HypergraphSpec(500, 1000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=3)
WIDE = synth.HypergraphSpec(240, 220, 2, 60, "uniform", 0.0, "uniform", 0.0, seed=4)
ZIPF_5K = synth.HypergraphSpec(2500, 5000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=8)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _graphs():
    out = {"tiny": (synth.TINY.n_nodes, *synth.generate(synth.TINY)),
           "zipf_small": (ZIPF_SMALL.n_nodes, *synth.generate(ZIPF_SMALL)),
           "wide": (WIDE.n_nodes, *synth.generate(WIDE)),
           "zipf5k": (ZIPF_5K.n_nodes, *synth.generate(ZIPF_5K))}
    for s in range(3):
        sets = _util.micro_graph(500 + s, n_nodes=12 + s, n_edges=25 + 3 * s, s_max=6)
        out[f"micro{s}"] = (12 + s, *_util.csr_from_sets(sets))
    sets = _util.micro_graph(600, n_nodes=70, n_edges=30, s_max=50)
    out["big0"] = (70, *_util.csr_from_sets(sets))
    return out


GRAPHS = _graphs()


# budgets: 1 byte (no bitmap: every node through its list), the default,
# and room for a bitmap of every node of degree >= E/1024
@pytest.mark.parametrize("budget", [1, 0, 1 << 30])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_onthefly_matches_oracle_aplus(name, budget):
    n, off, nodes = GRAPHS[name]
    samples = 3000 if name != "zipf5k" else 1500
    with B.Context() as c:
        c.load(n, off, nodes)
        got = c.count_sampled_onthefly(samples, 41, budget)
    ref = oracle.count_sampled(off, nodes, oracle.A_PLUS, samples, 41)
    for a, b in zip(got[:4], ref):
        assert np.array_equal(a, b)
    assert got[4] == oracle.project(off, nodes)[0]


def test_onthefly_other_theta():
    n, off, nodes = GRAPHS["zipf_small"]
    with B.Context(theta=2) as c:
        c.load(n, off, nodes)
        got = c.count_sampled_onthefly(2000, 3)
    ref = oracle.count_sampled(off, nodes, oracle.A_PLUS, 2000, 3, theta=2)
    for a, b in zip(got[:4], ref):
        assert np.array_equal(a, b)


def test_onthefly_keeps_its_structures_until_the_next_load():
    n, off, nodes = GRAPHS["zipf_small"]
    with B.Context() as c:
        c.load(n, off, nodes)
        first = c.count_sampled_onthefly(1000, 5, 1)
        again = c.count_sampled_onthefly(1000, 5, 1 << 30)     # budget ignored now
        assert all(np.array_equal(a, b) for a, b in zip(first[:4], again[:4]))
        n2, off2, nodes2 = GRAPHS["tiny"]
        c.load(n2, off2, nodes2)
        other = c.count_sampled_onthefly(1000, 5)
        ref = oracle.count_sampled(off2, nodes2, oracle.A_PLUS, 1000, 5)
        assert np.array_equal(other[1], ref[1])


def test_onthefly_errors():
    with B.Context() as c:
        with pytest.raises(B.MochyError):
            c.count_sampled_onthefly(10, 1)                     # nothing loaded
        c.load(3, np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32))
        with pytest.raises(B.MochyError) as e:
            c.count_sampled_onthefly(10, 1)                     # no hyperwedge
        assert e.value.code == B.E_INVALID
        n, off, nodes = GRAPHS["tiny"]
        c.load(n, off, nodes)
        with pytest.raises(B.MochyError):
            c.count_sampled_onthefly(0, 1)


def test_onthefly_matches_projected_on_medium():
    """The bench graph: 200,000 draws without the line graph equal the
    projected MoCHy-A+ on the same draws; |wedges| is half the sum of the
    oracle's line degrees."""
    off, nodes = synth.generate(synth.MEDIUM)
    deg = oracle.line_degrees(off, nodes)
    with B.Context() as c:
        c.load(synth.MEDIUM.n_nodes, off, nodes)
        fly = c.count_sampled_onthefly(200_000, 77)
        assert fly[4] == int(deg.sum()) // 2
        c.project()
        proj = c.count_sampled(B.MOCHY_A_PLUS, 200_000, 77)
    for a, b in zip(fly[:4], proj):
        assert np.array_equal(a, b)
    assert fly[0].sum() > 0
