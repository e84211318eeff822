"""The default (split) exact kernel against the oracle on the paths it runs at
full size (needs a GB300).

The small graphs of test_gpu_parity.py keep every dense row inside one chunk
of 32 words.  Here the dense threshold is forced low on graphs of 6,000 to
8,000 hyperedges, so that:

* more than 4,096 rows are dense (more than four 32-word chunks per overlap
  plane), and the next chunk's words are loaded ahead across chunks;
* nodes lie in 32 or more dense hyperedges (heavy-node bitmaps over several
  chunks) beside light nodes with short dense lists;
* a warp meets more than 8 hyperwedge signatures in a row (slots evicted),
  which a planted cluster of small hyperedges from a 24-node pool causes;
* a planted cluster of wide hyperedges from a 40-node pool gives overlaps of
  7 or more and triple intersections of 8 or more (the node-list fallback);

and the 26 h-motif and 431 3h-motif counts must equal the oracle's as int64.
The kernel's trace counters show that each path ran.

The medium bench workload itself (100,000 nodes, 200,000 hyperedges,
4.2e13 instances) is too large for the oracle to count whole; there the
shares of a seeded sample of rows (mochy_count_exact_rows: a row's neighbour
pairs as if open, plus the closed instances it owns in the split order
minus their as-if-open terms) must equal the oracle's shares under the same
order, and the full count must satisfy open + 3 closed = sum_e C(|N_e|, 2)
with line degrees from the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2310_15668_gb300 import binding as B, synth

pytestmark = pytest.mark.gpu


def _zipf6k():
    s = synth.HypergraphSpec(3000, 6000, 2, 25, "powerlaw", 2.5, "zipf", 0.7, seed=11)
    return s.n_nodes, *synth.generate(s)


def _zipf8k():
    s = synth.HypergraphSpec(6000, 8000, 2, 25, "powerlaw", 2.5, "zipf", 0.7, seed=12)
    return s.n_nodes, *synth.generate(s)


def _zipf6k_clusters():
    """zipf6k plus two planted clusters: 600 hyperedges of 2 to 9 nodes from a
    24-node pool (overlaps of 1 to 4 with every size, so a row meets many
    hyperwedge signatures) and 300 hyperedges of 14 to 25 nodes from a
    40-node pool (overlaps of 7 or more, triple intersections of 8 or more)."""
    n, off, nodes = _zipf6k()
    off, nodes = synth.plant_cluster(off, nodes, 600, 200, 24, 2, 9, seed=22)
    off, nodes = synth.plant_cluster(off, nodes, 300, 100, 40, 14, 25, seed=21)
    return n, off, nodes


# name: (graph, forced dense threshold)
GRAPHS = {"zipf6k": (_zipf6k, 32), "zipf8k": (_zipf8k, 16),
          "zipf6k_clusters": (_zipf6k_clusters, 32)}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


_cache = {}


def _graph(name):
    if name not in _cache:
        _cache[name] = GRAPHS[name][0]()
    return _cache[name]


def _oracle_counts(name, theta=1):
    key = (name, theta)
    if key not in _cache:
        _, off, nodes = _graph(name)
        _cache[key] = oracle.count_exact_threads(off, nodes, theta=theta, threads=0)
    return _cache[key]


def _split_rank(deg, thr):
    """The split kernel's order of hyperedges as int64 keys: rows of line
    degree below thr by id, then the others by (line degree, id)."""
    e = deg.size
    ids = np.arange(e, dtype=np.int64)
    return np.where(deg < thr, ids, (1 + deg.astype(np.int64)) * e + ids)


@pytest.mark.parametrize("rest_path", [1, 2])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_split_kernel_matches_oracle_on_multichunk_graphs(name, rest_path):
    """rest_path 1: each lane classifies the remaining candidates of its own
    word (the path of large hypergraphs); 2: they are spread over the warp."""
    n, off, nodes = _graph(name)
    thr = GRAPHS[name][1]
    with B.Context(dense_threshold=thr, rest_path=rest_path) as c:
        c.load(n, off, nodes)
        c.project()
        B.mochy_trace(c.h, 2)
        h, h3 = c.count_exact()
        tr = B.mochy_trace_read(c.h)
    oh, o3 = _oracle_counts(name)
    assert np.array_equal(h3, o3)
    assert np.array_equal(h, oh)
    # the paths this graph is here for
    assert tr["dense_threshold"] == thr
    assert tr["dense_rows"] >= 4096 and tr["dense_words"] >= 128      # four chunks or more
    assert tr["heavy_nodes"] > 0 and tr["heavy_bitmaps"] > 0
    assert tr["light_nodes"] > 0
    assert tr["table_candidates"] > 0
    if name == "zipf6k_clusters":
        assert tr["slots_evicted"] > 0
        assert tr["exact_candidates"] > 0


@pytest.mark.parametrize("rest_path", [1, 2])
def test_split_kernel_other_theta_on_multichunk_graph(rest_path):
    """theta = 2: the size-class bins of the kernel's other variant."""
    n, off, nodes = _graph("zipf6k_clusters")
    with B.Context(theta=2, dense_threshold=32, rest_path=rest_path) as c:
        c.load(n, off, nodes)
        c.project()
        h, h3 = c.count_exact()
    oh, o3 = _oracle_counts("zipf6k_clusters", theta=2)
    assert np.array_equal(h3, o3) and np.array_equal(h, oh)


@pytest.mark.parametrize("name", ["zipf6k", "zipf6k_clusters"])
def test_split_rows_match_oracle_under_the_split_order(name):
    """Row shares of the split kernel (pairs of a row's neighbours as if
    open, plus the closed instances it owns in the split order minus their
    as-if-open terms) equal the oracle's shares under the same order; the
    parts of a partition of all rows add up to the full count."""
    n, off, nodes = _graph(name)
    thr = GRAPHS[name][1]
    deg = oracle.line_degrees(off, nodes)
    rank = _split_rank(deg, thr)
    e = deg.size
    rng = np.random.default_rng(3)
    with B.Context(dense_threshold=thr) as c:
        c.load(n, off, nodes)
        c.project()
        dense = np.flatnonzero(deg >= thr)
        sparse = np.flatnonzero(deg < thr)
        rows = np.concatenate([rng.choice(dense, 60, replace=False),
                               rng.choice(sparse, min(20, sparse.size), replace=False)])
        rows = rows.astype(np.int32)
        g = c.count_exact_rows(rows)
        o = oracle.count_split_rows(off, nodes, rows, rank, threads=0)
        assert np.array_equal(g[0], o[0]) and np.array_equal(g[1], o[1])
        parts = np.array_split(rng.permutation(e).astype(np.int32), 3)
        acc = sum(c.count_exact_rows(p)[1] for p in parts)
        assert np.array_equal(acc, c.count_exact()[1])
        assert c.count_exact_rows(np.zeros(0, np.int32))[1].sum() == 0


# the tuner's threshold on the medium workload (143,930 dense rows, 4,498
# words per overlap plane); the test checks that the tuner still picks it
MEDIUM_THRESHOLD = 1024


@pytest.fixture(scope="module")
def medium():
    off, nodes = synth.generate(synth.MEDIUM)
    deg = oracle.line_degrees(off, nodes)
    return off, nodes, deg


def test_medium_full_count_degree_identity(medium):
    """The bench configuration itself, counted whole by the default kernel:
    open instances plus three times the closed ones are the pairs of
    neighbours of all hyperedges, with |N_e| from the oracle."""
    off, nodes, deg = medium
    T = oracle.tables()
    with B.Context() as c:
        c.load(synth.MEDIUM.n_nodes, off, nodes)
        c.project()
        B.mochy_trace(c.h, 2)
        h, h3 = c.count_exact()
        tr = B.mochy_trace_read(c.h)
    assert tr["dense_threshold"] == MEDIUM_THRESHOLD
    opened = int(sum(int(h[t]) for t in range(26) if T["h_open"][t]))
    closed = int(h.sum()) - opened
    assert opened + 3 * closed == int((deg * (deg - 1) // 2).sum())
    merged = np.zeros(26, np.int64)
    np.add.at(merged, T["t_to_h"] - 1, h3)
    assert np.array_equal(merged, h)
    # every path of the dense kernel ran on this workload
    assert tr["slots_evicted"] > 0 and tr["slots_flushed_full"] > 0
    assert tr["exact_candidates"] > 0 and tr["table_candidates"] > 0


def test_medium_rows_match_oracle(medium):
    """Seeded rows of the medium workload: sparse rows, dense rows of line
    degree up to 4,000 (their hyperwedges scan the full 4,498-word planes) and
    two of degree 10,000 to 14,000, counted by the split kernel at the
    tuner's threshold and by the oracle under the same order."""
    off, nodes, deg = medium
    rank = _split_rank(deg, MEDIUM_THRESHOLD)
    rng = np.random.default_rng(17)
    sparse = np.flatnonzero(deg < MEDIUM_THRESHOLD)
    mid = np.flatnonzero((deg >= MEDIUM_THRESHOLD) & (deg <= 4000))
    big = np.flatnonzero((deg >= 10_000) & (deg <= 14_000))
    rows = np.concatenate([rng.choice(sparse, 24, replace=False),
                           rng.choice(mid, 40, replace=False),
                           rng.choice(big, 2, replace=False)]).astype(np.int32)
    with B.Context(dense_threshold=MEDIUM_THRESHOLD) as c:
        c.load(synth.MEDIUM.n_nodes, off, nodes)
        c.project()
        B.mochy_trace(c.h, 2)
        g = c.count_exact_rows(rows)
        tr = B.mochy_trace_read(c.h)
    o = oracle.count_split_rows(off, nodes, rows, rank, threads=0)
    assert np.array_equal(g[1], o[1])
    assert np.array_equal(g[0], o[0])
    assert tr["dense_rows_counted"] == 42
    assert g[1].any()


def test_measured_tuner_keeps_the_fastest_threshold_and_counts_stay_exact():
    n, off, nodes = _graph("zipf6k")
    with B.Context() as c:
        c.load(n, off, nodes)
        c.project()
        best, tried = B.mochy_tune_dense_threshold(c.h, [16, 32, 64, 128], 0.05, 3)
        assert [t for t, _ in tried] == [16, 32, 64, 128]
        assert all(ms > 0 for _, ms in tried)
        assert best == min(tried, key=lambda x: x[1])[0]
        B.mochy_trace(c.h, 1)
        h, h3 = c.count_exact()
        assert B.mochy_trace_read(c.h)["dense_threshold"] == best
        best2, tried2 = B.mochy_tune_dense_threshold(c.h)        # the model's five
        assert len(tried2) == 5 and best2 in [t for t, _ in tried2]
    oh, o3 = _oracle_counts("zipf6k")
    assert np.array_equal(h3, o3) and np.array_equal(h, oh)
