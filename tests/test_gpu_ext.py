"""kh-motifs, instance enumeration and radial node profiles on the GPU against
the oracle, through the C ABI (needs a GB300).

kh-motif counts (Section 4.1 "Extensions Beyond Ternary") and their
patterns must equal the oracle's as int64 / exactly; the enumerated
instances (Algorithm "alg:enum") must be the oracle's rows, compared as sets
(the device writes them in no particular order, and each exactly once);
radial node profiles (Section 3.1) must equal the oracle's rows as int64.
"""
import numpy as np
import pytest

import oracle
from paper_2310_15668_gb300 import binding as B, synth
from tests import _util

pytestmark = pytest.mark.gpu

ZIPF_SMALL = synth.HypergraphSpec(500, 1000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=3)
WIDE = synth.HypergraphSpec(240, 220, 2, 60, "uniform", 0.0, "uniform", 0.0, seed=4)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _graphs():
    out = {"tiny": (synth.TINY.n_nodes, *synth.generate(synth.TINY)),
           "zipf_small": (ZIPF_SMALL.n_nodes, *synth.generate(ZIPF_SMALL)),
           "wide": (WIDE.n_nodes, *synth.generate(WIDE))}
    for s in range(6):
        sets = _util.micro_graph(500 + s, n_nodes=12 + s, n_edges=25 + 3 * s, s_max=6)
        out[f"micro{s}"] = (12 + s, *_util.csr_from_sets(sets))
    for s in range(2):
        sets = _util.micro_graph(600 + s, n_nodes=70, n_edges=30, s_max=50)
        out[f"big{s}"] = (70, *_util.csr_from_sets(sets))
    return out


GRAPHS = _graphs()


@pytest.fixture(scope="module")
def ctx():
    with B.Context() as c:
        yield c


def test_4h_patterns_match_oracle(ctx):
    K = oracle.kh_tables(4)
    assert K["to_h"].size == 3076
    for i in range(1, 3077):
        assert np.array_equal(B.mochy_kh_pattern(ctx.h, 4, i), K["pattern"][i - 1])
    with pytest.raises(B.MochyError):
        B.mochy_kh_pattern(ctx.h, 4, 3077)


@pytest.mark.parametrize("k,thr", [(4, (1, 2)), (4, (2, 4)), (3, (1,)), (3, (2,)), (2, ())])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_kh_counts_match_oracle(ctx, name, k, thr):
    n, off, nodes = GRAPHS[name]
    ctx.load(n, off, nodes)
    ctx.project()
    h, kh = ctx.count_kh(k, thr)
    oh, okh = oracle.count_exact_kh(off, nodes, k, thr)
    assert np.array_equal(kh, okh)
    assert np.array_equal(h, oh)
    if k == 3:
        # the 3h-motifs of theta = thr[0], by the regular count
        with B.Context(theta=thr[0]) as c3:
            c3.load(n, off, nodes)
            c3.project()
            assert np.array_equal(c3.count_exact()[1], kh)


def test_kh_bad_arguments(ctx):
    n, off, nodes = GRAPHS["micro1"]
    ctx.load(n, off, nodes)
    ctx.project()
    for k, thr in ((4, (2, 2)), (4, (0, 3)), (3, (64,))):
        with pytest.raises(B.MochyError) as e:
            ctx.count_kh(k, thr)
        assert e.value.code == B.E_INVALID
    with pytest.raises(B.MochyError) as e:
        ctx.count_kh(5, (1, 2, 3))
    assert e.value.code == B.E_UNSUPPORTED


def _sorted_rows(rows):
    """Rows in ascending (i, j, k) order (the triple identifies the row)."""
    return rows[np.lexsort((rows[:, 2], rows[:, 1], rows[:, 0]))]


@pytest.mark.parametrize("name", ["tiny", "wide", "micro2", "big1"])
def test_enumeration_matches_oracle(ctx, name):
    n, off, nodes = GRAPHS[name]
    ctx.load(n, off, nodes)
    ctx.project()
    want, n_want = oracle.enumerate_instances(off, nodes)
    got, n_got = ctx.enumerate(n_want + 10)
    assert n_got == n_want == got.shape[0]
    g = _sorted_rows(got)
    # each instance once: no two rows with the same triple
    assert not (g[1:, :3] == g[:-1, :3]).all(axis=1).any()
    assert np.array_equal(g, _sorted_rows(want))


def test_enumeration_with_small_capacity(ctx):
    n, off, nodes = GRAPHS["tiny"]
    ctx.load(n, off, nodes)
    ctx.project()
    want, n_want = oracle.enumerate_instances(off, nodes)
    got, n_got = ctx.enumerate(1000)
    assert n_got == n_want and got.shape == (1000, 5)
    known = {tuple(int(v) for v in r) for r in want}
    assert all(tuple(int(v) for v in r) in known for r in got)
    none, n0 = ctx.enumerate(0)
    assert n0 == n_want and none.shape[0] == 0


@pytest.mark.parametrize("name", ["micro0", "micro3", "micro5", "big0", "big1", "zipf_small"])
def test_radial_profiles_match_oracle(ctx, name):
    n, off, nodes = GRAPHS[name]
    ctx.load(n, off, nodes)
    ctx.project()
    gh, g3 = ctx.radial_node_profile()
    oh, o3 = oracle.radial_node_profile(n, off, nodes)
    assert np.array_equal(g3, o3)
    assert np.array_equal(gh, oh)
    sh, s3 = ctx.star_node_profile()
    assert (g3 >= s3).all()
