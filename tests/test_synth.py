"""The seeded input generator (paper_2310_15668_gb300/synth.py).

Every workload comes from it, so its recipe is pinned here: the same spec
always gives the same hypergraph; hyperedges are distinct sets of distinct
in-range nodes, sorted, with sizes in [s_min, s_max]; sizes follow the
stated law (truncated power law s^-alpha or uniform), members the stated
node popularity (Zipf: frequency proportional to 1/rank), and batch sizes
are log-uniform in [lo, hi].
"""
import math

import numpy as np

from paper_2310_15668_gb300 import synth


def _rows(off, nodes):
    return [nodes[off[i]:off[i + 1]] for i in range(off.size - 1)]


def test_same_spec_same_hypergraph_and_seeds_differ():
    spec = synth.HypergraphSpec(300, 600, 2, 8, "powerlaw", 2.5, "zipf", 1.0, seed=11)
    a = synth.generate(spec)
    b = synth.generate(spec)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = synth.generate(synth.HypergraphSpec(300, 600, 2, 8, "powerlaw", 2.5, "zipf", 1.0,
                                            seed=12))
    assert not (np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]))


def test_hyperedges_are_distinct_sorted_sets_in_range():
    for spec in (synth.TINY,
                 synth.HypergraphSpec(500, 3000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=3)):
        off, nodes = synth.generate(spec)
        assert off[0] == 0 and off.size == spec.n_edges + 1 and (np.diff(off) > 0).all()
        assert nodes.min() >= 0 and nodes.max() < spec.n_nodes
        seen = set()
        for r in _rows(off, nodes):
            assert spec.s_min <= r.size <= spec.s_max
            assert (np.diff(r) > 0).all()                  # sorted, no repeated node
            seen.add(tuple(r.tolist()))
        assert len(seen) == spec.n_edges


def test_size_law():
    # many nodes and uniform members, so that duplicates (dropped) are rare
    spec = synth.HypergraphSpec(200_000, 40_000, 2, 25, "powerlaw", 2.5, "uniform", 0.0, seed=5)
    off, _ = synth.generate(spec)
    sizes = np.diff(off)
    s = np.arange(2, 26)
    p = s ** -2.5
    p /= p.sum()
    freq = np.bincount(sizes, minlength=26)[2:26] / sizes.size
    for i in range(4):                                     # the well-populated sizes
        assert abs(freq[i] - p[i]) < 4 * math.sqrt(p[i] * (1 - p[i]) / sizes.size) + 1e-3
    u = synth.HypergraphSpec(1000, 5000, 2, 5, "uniform", 0.0, "uniform", 0.0, seed=6)
    f = np.bincount(np.diff(synth.generate(u)[0]), minlength=6)[2:6] / 5000
    assert np.all(np.abs(f - 0.25) < 0.03)


def test_zipf_popularity():
    # frequency proportional to rank^-s: the log-log slope over the middle
    # ranks is -s (the top ranks are flattened a little by drawing members
    # without replacement and by dropping repeated hyperedges)
    spec = synth.HypergraphSpec(50_000, 40_000, 3, 3, "uniform", 0.0, "zipf", 1.0, seed=8)
    _, nodes = synth.generate(spec)
    cnt = np.bincount(nodes, minlength=spec.n_nodes).astype(np.float64)
    ranks = np.arange(10, 1000)
    slope = np.polyfit(np.log(ranks + 1), np.log(np.maximum(cnt[ranks], 0.5)), 1)[0]
    assert abs(slope + 1.0) < 0.1
    u = synth.HypergraphSpec(1000, 5000, 3, 3, "uniform", 0.0, "uniform", 0.0, seed=8)
    cu = np.bincount(synth.generate(u)[1], minlength=1000)
    assert cu.max() < 2 * cu.mean() and cu.min() > 0.3 * cu.mean()


def test_batch_sizes_are_log_uniform():
    es = np.array([synth.loguniform_edges(4, i, 2000, 20000) for i in range(4000)])
    assert es.min() >= 2000 and es.max() <= 20000
    logs = np.log(es)
    assert abs(logs.mean() - 0.5 * (math.log(2000) + math.log(20000))) < 0.05
    spec = synth.batch_spec(4, 3, 2000, 20000)
    assert spec.n_nodes == max(spec.n_edges // 2, 64) and spec.s_max == 25


def test_named_workloads():
    assert synth.TINY.describe() == "N=1000 E=2000 sizes U[2,5] members uniform seed 0"
    assert synth.MEDIUM.describe() == ("N=100000 E=200000 sizes s^-2.5 on [2,25] members "
                                       "Zipf(1.0) seed 1")
    assert (synth.LARGE.n_nodes, synth.LARGE.n_edges, synth.LARGE.zipf_s) == (1_500_000,
                                                                              2_500_000, 1.1)
