"""Batched significance/CP (mochy_profile_batch) on the GPU, through the C ABI.

Every hypergraph of a batch must get exactly what it gets alone: counts of
the input and of each randomized copy equal as int64 to the oracle's and to
mochy_profile's, significances and CPs within 1e-12 relative of the oracle
and identical to mochy_profile's (same device arithmetic).  Batches mix
sizes, include a hypergraph without hyperedges, force dense rows (small
dense threshold) so that several hypergraphs share the dense bitmap word
space, and run in several waves (smaller unions).
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


def _zipf(n_edges, seed, s_max=25):
    spec = synth.HypergraphSpec(max(n_edges // 2, 64), n_edges, 2, s_max, "powerlaw", 2.5,
                                "zipf", 1.0, seed=seed)
    off, nodes = synth.generate(spec)
    return spec.n_nodes, off, nodes


def _mixed_batch():
    gs = [_zipf(300, 11), (synth.TINY.n_nodes, *synth.generate(synth.TINY)), _zipf(1200, 12),
          (5, np.zeros(1, np.int64), np.zeros(0, np.int32))]
    sets = _util.micro_graph(77, n_nodes=30, n_edges=40, s_max=8)
    gs.append((30, *_util.csr_from_sets(sets)))
    sets = _util.micro_graph(78, n_nodes=70, n_edges=30, s_max=50)
    gs.append((70, *_util.csr_from_sets(sets)))
    return gs


def _cfg(**kw):
    cfg = B.mochy_config_default()
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


@pytest.mark.parametrize("thr", [0, 16])
def test_batch_matches_oracle(thr):
    gs = _mixed_batch()
    R = 3
    seeds = [5 + 7 * g for g in range(len(gs))]
    sig_h, cp_h, sig_3h, cp_3h, ch, c3, deg, info = B.mochy_profile_batch(
        gs, R, seeds, _cfg(dense_threshold=thr))
    assert info["n_units"] == len(gs) * (R + 1) and info["n_waves"] == 1
    for g, (n, off, nodes) in enumerate(gs):
        o = oracle.profile(n, off, nodes, R, seeds[g])
        assert np.array_equal(ch[g], o["counts_h"]), g
        assert np.array_equal(c3[g], o["counts_3h"]), g
        for got, key in ((sig_h, "sig_h"), (cp_h, "cp_h"), (sig_3h, "sig_3h"), (cp_3h, "cp_3h")):
            np.testing.assert_allclose(got[g], o[key], rtol=1e-12, atol=1e-300)
        assert deg[g] == (1 if (o["degenerate"][0] or o["degenerate"][1]) else 0)
    assert info["instances"] == int(ch.sum())


def test_batch_equals_one_at_a_time():
    gs = [_zipf(e, 20 + i) for i, e in enumerate((800, 2500, 1500, 4000, 600))]
    R = 4
    seeds = [101 + g for g in range(len(gs))]
    for thr in (0, 24):
        sig_h, cp_h, sig_3h, cp_3h, ch, c3, deg, info = B.mochy_profile_batch(
            gs, R, seeds, _cfg(dense_threshold=thr))
        for g, (n, off, nodes) in enumerate(gs):
            with B.Context(dense_threshold=thr) as c:
                c.load(n, off, nodes)
                one = c.profile(R, seeds[g])
            assert np.array_equal(ch[g], one["counts_h"]), (thr, g)
            assert np.array_equal(c3[g], one["counts_3h"]), (thr, g)
            assert np.array_equal(sig_h[g], one["sig_h"]) and np.array_equal(cp_h[g], one["cp_h"])
            assert np.array_equal(sig_3h[g], one["sig_3h"])
            assert np.array_equal(cp_3h[g], one["cp_3h"])
        assert info["ms_count"] > 0.0


def test_batch_in_waves(monkeypatch):
    gs = [_zipf(e, 40 + i) for i, e in enumerate((400, 700, 500, 900, 300))]
    R = 2
    seeds = [9] * len(gs)
    whole = B.mochy_profile_batch(gs, R, seeds)
    monkeypatch.setenv("MOCHY_BATCH_MAX_GRAPHS", "2")
    waves = B.mochy_profile_batch(gs, R, seeds)
    assert waves[7]["n_waves"] == 3 and whole[7]["n_waves"] == 1
    for a, b in zip(whole[:7], waves[:7]):
        assert np.array_equal(a, b)


def test_batch_errors():
    g = _zipf(200, 3)
    with pytest.raises(B.MochyError) as e:
        B.mochy_profile_batch([], 2, [])
    assert e.value.code == B.E_INVALID
    with pytest.raises(B.MochyError) as e:
        B.mochy_profile_batch([g], 2, [1], _cfg(exact_kernel=1))
    assert e.value.code == B.E_UNSUPPORTED
    n, off, nodes = g
    bad = nodes.copy()
    bad[0] = n                                   # node id out of range
    with pytest.raises(B.MochyError) as e:
        B.mochy_profile_batch([g, (n, off, bad)], 2, [1, 2])
    assert e.value.code == B.E_INVALID
    with pytest.raises(B.MochyError) as e:
        B.mochy_profile_batch([g], 0, [1])
    assert e.value.code == B.E_INVALID
