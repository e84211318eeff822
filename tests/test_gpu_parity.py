"""GPU path against the oracle, through the C ABI (needs a GB300).

Exact counts must match bit for bit as int64; sampled raw counts and their
FP64 estimates must match bit for bit on the same Philox draws; randomized
copies must be identical hypergraphs; CPs agree to 1e-12 relative.
"""
import functools

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


@pytest.fixture(scope="module")
def ctx():
    with B.Context() as c:
        yield c


def _graphs():
    out = {"tiny": (synth.TINY.n_nodes, *synth.generate(synth.TINY)),
           "zipf_small": (ZIPF_SMALL.n_nodes, *synth.generate(ZIPF_SMALL)),
           "wide": (WIDE.n_nodes, *synth.generate(WIDE))}
    for s in range(12):
        sets = _util.micro_graph(500 + s, n_nodes=12 + s, n_edges=25 + 3 * s, s_max=6)
        out[f"micro{s}"] = (12 + s, *_util.csr_from_sets(sets))
    for s in range(4):
        sets = _util.micro_graph(600 + s, n_nodes=70, n_edges=30, s_max=50)
        out[f"big{s}"] = (70, *_util.csr_from_sets(sets))
    return out


GRAPHS = _graphs()


@functools.lru_cache(maxsize=None)
def _oracle_exact(name, theta=1):
    n, off, nodes = GRAPHS[name]
    return oracle.count_exact(off, nodes, theta=theta)


def test_motif_numbering_matches_oracle(ctx):
    T = oracle.tables()
    for hid in range(1, 27):
        assert list(B.mochy_motif_pattern(2, hid)) == list(T["h_pattern"][hid - 1])
    for tid in range(1, 432):
        assert list(B.mochy_motif_pattern(3, tid)) == list(T["t_pattern"][tid - 1])


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_load_and_project(ctx, name):
    n, off, nodes = GRAPHS[name]
    ctx.load(n, off, nodes)
    _, goff, gnodes = ctx.hypergraph()
    ooff, onodes, _ = oracle.dedupe(off, nodes)
    assert np.array_equal(goff, ooff) and np.array_equal(gnodes, onodes)
    nw, md = ctx.project()
    onw, omd, odeg = oracle.project(off, nodes)
    assert (nw, md) == (onw, omd)
    assert np.array_equal(ctx.line_degrees(), odeg)


# exact-count kernels: the per-hyperwedge scan, and the split kernel with the
# tuned threshold, with (nearly) every row dense, and with a middle threshold
VARIANTS = {"scan": dict(exact_kernel=1), "split": dict(), "dense": dict(dense_threshold=2),
            "mixed": dict(dense_threshold=24),
            # the same with the dense rows' remaining candidates taken per lane
            # (small hypergraphs spread them over the warp by default)
            "dense_lane": dict(dense_threshold=2, rest_path=1),
            "mixed_lane": dict(dense_threshold=24, rest_path=1)}


@pytest.fixture(scope="module")
def variant_ctx():
    ctxs = {k: B.Context(**v) for k, v in VARIANTS.items()}
    yield ctxs
    for c in ctxs.values():
        c.close()


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_exact_counts(variant_ctx, name, variant):
    c = variant_ctx[variant]
    n, off, nodes = GRAPHS[name]
    c.load(n, off, nodes)
    c.project()
    h, h3 = c.count_exact()
    oh, o3 = _oracle_exact(name)
    assert np.array_equal(h3, o3)
    assert np.array_equal(h, oh)


def test_split_matches_scan_on_larger_zipf_graph(variant_ctx):
    """GPU against GPU where the oracle is too slow: 20,000 hyperedges with a
    hub of about 4,500 hyperedges; every kernel variant gives the same counts,
    and the open/closed totals satisfy the line-graph degree identity."""
    spec = synth.HypergraphSpec(10_000, 20_000, 2, 25, "powerlaw", 2.5, "zipf", 1.0, seed=5)
    off, nodes = synth.generate(spec)
    res = {}
    for v, c in variant_ctx.items():
        c.load(spec.n_nodes, off, nodes)
        c.project()
        res[v] = c.count_exact()
    for v in res:
        assert np.array_equal(res[v][1], res["scan"][1]), v
    T = oracle.tables()
    h = res["split"][0]
    deg = variant_ctx["split"].line_degrees()
    op = int(sum(h[t] for t in range(26) if T["h_open"][t]))
    assert op + 3 * (int(h.sum()) - op) == int((deg * (deg - 1) // 2).sum())


@pytest.mark.parametrize("theta", [2, 3])
@pytest.mark.parametrize("variant", ["scan", "split", "dense", "dense_lane"])
@pytest.mark.parametrize("name", ["wide", "zipf_small"])
def test_exact_counts_other_theta(theta, variant, name):
    n, off, nodes = GRAPHS[name]
    with B.Context(theta=theta, **VARIANTS[variant]) as c:
        c.load(n, off, nodes)
        c.project()
        h, h3 = c.count_exact()
    oh, o3 = _oracle_exact(name, theta)
    assert np.array_equal(h3, o3) and np.array_equal(h, oh)


def test_duplicates_are_dropped(ctx):
    sets = [[3, 1, 2], [2, 3, 1], [5], [1, 2, 4], [4, 5], [5], [1, 2, 3]]
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in sets])
    nodes = np.array([v for s in sets for v in s], np.int32)
    assert ctx.load(6, off, nodes) == 3
    _, goff, gnodes = ctx.hypergraph()
    ooff, onodes, _ = oracle.dedupe(off, nodes)
    assert np.array_equal(goff, ooff) and np.array_equal(gnodes, onodes)


@pytest.mark.parametrize("name", ["tiny", "zipf_small", "wide", "micro3", "big1"])
@pytest.mark.parametrize("method", [B.MOCHY_A, B.MOCHY_A_PLUS])
def test_sampled_bit_exact(ctx, name, method):
    n, off, nodes = GRAPHS[name]
    ctx.load(n, off, nodes)
    ctx.project()
    samples = (40 if name == "zipf_small" else 200) if method == B.MOCHY_A else 2000
    for seed in (1, 2**40 + 5):
        g = ctx.count_sampled(method, samples, seed)
        o = oracle.count_sampled(off, nodes, method, samples, seed)
        for a, b in zip(g, o):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["tiny", "zipf_small", "micro5", "micro9"])
def test_randomized_copy_identical(ctx, name):
    n, off, nodes = GRAPHS[name]
    ctx.load(n, off, nodes)
    for copy in (0, 7):
        with ctx.randomize(99, copy) as r:
            _, roff, rnodes = r.hypergraph()
        ooff, onodes = oracle.randomize(n, off, nodes, 99, copy)
        assert np.array_equal(roff, ooff) and np.array_equal(rnodes, onodes)


@pytest.mark.parametrize("name", ["micro2", "micro7", "tiny"])
def test_profile(ctx, name):
    n, off, nodes = GRAPHS[name]
    ctx.load(n, off, nodes)
    R = 3
    g = ctx.profile(R, 5)
    o = oracle.profile(n, off, nodes, R, 5)
    assert np.array_equal(g["counts_h"], o["counts_h"])
    assert np.array_equal(g["counts_3h"], o["counts_3h"])
    for key in ("sig_h", "cp_h", "sig_3h", "cp_3h"):
        np.testing.assert_allclose(g[key], o[key], rtol=1e-12, atol=1e-300)


def test_subset_matches_oracle(ctx):
    n, off, nodes = GRAPHS["zipf_small"]
    ctx.load(n, off, nodes)
    ctx.project()
    rng = np.random.default_rng(1)
    anchors = rng.choice(off.size - 1, size=40, replace=False).astype(np.int32)
    g = ctx.count_exact_subset(anchors)
    o = oracle.count_exact_subset(off, nodes, anchors)
    assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1])
    # all anchors together give the full count
    allh = ctx.count_exact_subset(np.arange(off.size - 1, dtype=np.int32))
    full = ctx.count_exact()
    assert np.array_equal(allh[1], full[1])


def test_errors(ctx):
    with pytest.raises(B.MochyError) as e:
        ctx.load(4, np.array([0, 2, 2], np.int64), np.array([0, 1], np.int32))
    assert e.value.code == B.E_INVALID                    # empty hyperedge
    with pytest.raises(B.MochyError) as e:
        ctx.load(4, np.array([0, 2], np.int64), np.array([0, 9], np.int32))
    assert e.value.code == B.E_INVALID                    # node out of range
    with pytest.raises(B.MochyError) as e:
        ctx.load(4, np.array([0, 2], np.int64), np.array([1, 1], np.int32))
    assert e.value.code == B.E_INVALID                    # repeated node
    with pytest.raises(B.MochyError) as e:
        ctx.load(100, np.array([0, 64], np.int64), np.arange(64, dtype=np.int32))
    assert e.value.code == B.E_UNSUPPORTED                # more than 63 nodes
    ctx.load(4, np.array([0, 2, 4], np.int64), np.array([0, 1, 1, 2], np.int32))
    with pytest.raises(B.MochyError) as e:
        ctx.count_exact()
    assert e.value.code == B.E_NOT_PROJECTED
    with pytest.raises(B.MochyError) as e:
        ctx.count_sampled(B.MOCHY_A_PLUS, 0, 1)
    with B.Context(budget=200 << 10) as small:
        n, off, nodes = GRAPHS["tiny"]
        with pytest.raises(B.MochyError) as e:
            small.load(n, off, nodes)
            small.project()
        assert e.value.code == B.E_NOMEM


def test_empty_graphs(ctx):
    ctx.load(3, np.zeros(1, np.int64), np.zeros(0, np.int32))
    assert ctx.project() == (0, 0)
    h, h3 = ctx.count_exact()
    assert h.sum() == 0 and h3.sum() == 0
    ctx.load(3, np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32))
    assert ctx.project() == (0, 0)
    assert ctx.count_exact()[0].sum() == 0
