"""Pins of the oracle's MoCHy-A+ without the line graph (CPU only;
Section 3.4 "Motif Counting without Line Graphs", Algorithms "alg_memdeg"
and "alg_memdeg_adv").

Memoization only decides which neighbourhoods are rebuilt, so at every
budget, from nothing to the whole line graph, both on-the-fly algorithms
must classify exactly what MoCHy-A+ on the projected line graph classifies
from the same Philox draws: raw counts and FP64 estimates bit-equal.  The
projected MoCHy-A+ is itself pinned in test_oracle_sampling.py.
"""
import numpy as np
import pytest

import oracle
from paper_2310_15668_gb300 import synth

ZIPF = synth.HypergraphSpec(500, 1000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=3)


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("frac", [0.0, 0.01, 0.1, 0.5, 1.0])
@pytest.mark.parametrize("spec", [synth.TINY, ZIPF], ids=["tiny", "zipf"])
def test_onthefly_equals_projected_at_every_budget(spec, frac, method):
    off, nodes = synth.generate(spec)
    nw, _, _ = oracle.project(off, nodes)
    ref = oracle.count_sampled(off, nodes, oracle.A_PLUS, 1500, 23)
    got = oracle.count_aplus_onthefly(off, nodes, method, 1500, 23, int(frac * 2 * nw))
    for a, b in zip(got[:4], ref):
        assert np.array_equal(a, b)
    built, evicted, wedges = (int(v) for v in got[4])
    assert wedges == nw
    if frac == 0.0:
        assert evicted == 0            # nothing is ever memoized
    if frac == 1.0:
        assert evicted == 0            # everything fits


def test_onthefly_other_theta():
    off, nodes = synth.generate(ZIPF)
    ref = oracle.count_sampled(off, nodes, oracle.A_PLUS, 800, 5, theta=2)
    for method in (1, 2):
        got = oracle.count_aplus_onthefly(off, nodes, method, 800, 5, 5000, theta=2)
        for a, b in zip(got[:4], ref):
            assert np.array_equal(a, b)


def test_whole_line_graph_budget_builds_each_neighbourhood_once():
    """With room for every neighbourhood nothing is rebuilt: the number of
    getNeighbors calls is the number of distinct hyperedges drawn."""
    off, nodes = synth.generate(ZIPF)
    nw, _, _ = oracle.project(off, nodes)
    for method in (1, 2):
        built = int(oracle.count_aplus_onthefly(off, nodes, method, 500, 9, 2 * nw)[4][0])
        again = int(oracle.count_aplus_onthefly(off, nodes, method, 500, 9, 4 * nw)[4][0])
        assert built == again and built <= 2 * 500
