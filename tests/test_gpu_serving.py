"""Serving with continuous batching (mochy_server_*) on the GPU, via the C ABI.

A mix of exact, sampled and profile requests submitted together must overlap
on the device (more than one in flight) and every result must equal the
result of the same calls made alone (exact and raw counts as int64,
estimates and CPs bit for bit: the device arithmetic is the same).  Under a
budget that admits one request at a time the results are unchanged; a
request larger than the whole budget and a submission to a full queue are
refused.
"""
import numpy as np
import pytest

from paper_2310_15668_gb300 import binding as B, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _zipf(n_edges, seed):
    spec = synth.HypergraphSpec(max(n_edges // 2, 64), n_edges, 2, 25, "powerlaw", 2.5, "zipf",
                                1.0, seed=seed)
    off, nodes = synth.generate(spec)
    return spec.n_nodes, off, nodes


def _estimate(n, off, nodes):
    # the server's admission estimate (line graph bound and per-element arrays)
    deg = np.bincount(nodes, minlength=n).astype(np.float64)
    w = float((0.5 * deg * (deg - 1)).sum())
    E, T = off.size - 1, int(off[-1])
    return int(16.0 * w + 96.0 * E + 48.0 * T + 16.0 * n) + (1 << 20)


def _alone(kind, g, samples=0, n_random=0, seed=0):
    n, off, nodes = g
    with B.Context() as c:
        c.load(n, off, nodes)
        c.project()
        if kind == B.MOCHY_REQ_EXACT:
            h, t = c.count_exact()
            return {"counts_h": h, "counts_3h": t}
        if kind == B.MOCHY_REQ_SAMPLED:
            rh, r3, eh, e3 = c.count_sampled(B.MOCHY_A_PLUS, samples, seed)
            return {"counts_h": rh, "counts_3h": r3, "est_h": eh, "est_3h": e3}
        p = c.profile(n_random, seed)
        return {"counts_h": p["counts_h"][0], "counts_3h": p["counts_3h"][0], "sig_h": p["sig_h"],
                "cp_h": p["cp_h"], "sig_3h": p["sig_3h"], "cp_3h": p["cp_3h"]}


def _mix():
    gs = [_zipf(e, 60 + i) for i, e in enumerate((3000, 800, 5000, 1500))]
    tiny = (synth.TINY.n_nodes, *synth.generate(synth.TINY))
    reqs = []
    for i, g in enumerate(gs):
        reqs.append((B.MOCHY_REQ_EXACT, g, dict()))
        reqs.append((B.MOCHY_REQ_SAMPLED, g, dict(samples=5000 + 100 * i, seed=30 + i)))
    reqs.append((B.MOCHY_REQ_PROFILE, tiny, dict(n_random=3, seed=5)))
    reqs.append((B.MOCHY_REQ_PROFILE, gs[1], dict(n_random=2, seed=6)))
    reqs.append((B.MOCHY_REQ_EXACT, tiny, dict()))
    return reqs


def _check_same(res, ref):
    assert res["status"] >= 0
    for k, v in ref.items():
        assert np.array_equal(res[k], v), k


def test_mix_overlaps_and_matches_alone():
    reqs = _mix()
    with B.Server(n_slots=4) as srv:
        tickets = [srv.submit(kind, *g, samples=kw.get("samples", 0),
                              n_random=kw.get("n_random", 0), seed=kw.get("seed", 0))
                   for kind, g, kw in reqs]
        results = []
        for t in tickets:
            r = None
            for _ in range(600):
                r = srv.poll(t, wait_ms=1000)
                if r is not None:
                    break
            assert r is not None
            results.append(r)
        st = srv.stats()
    bad = [(i, r["status"], r["error"]) for i, r in enumerate(results) if r["status"] < 0]
    assert not bad
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["peak_in_flight"] >= 2
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    for (kind, g, kw), r in zip(reqs, results):
        _check_same(r, _alone(kind, g, **kw))
        assert r["latency_ms"] >= r["service_ms"] > 0


def test_one_at_a_time_budget():
    g = _zipf(2000, 70)
    est = _estimate(*g)
    with B.Server(n_slots=4, budget=int(1.5 * est)) as srv:
        tickets = [srv.submit(B.MOCHY_REQ_EXACT, *g) for _ in range(4)]
        results = [srv.poll(t, wait_ms=120000) for t in tickets]
        st = srv.stats()
        with pytest.raises(B.MochyError) as e:           # larger than the whole budget
            srv.submit(B.MOCHY_REQ_EXACT, *_zipf(6000, 71))
        assert e.value.code == B.E_NOMEM
    assert st["peak_in_flight"] == 1 and st["peak_reserved_bytes"] <= int(1.5 * est)
    ref = _alone(B.MOCHY_REQ_EXACT, g)
    for r in results:
        _check_same(r, ref)


def test_queue_full_and_bad_requests():
    g = _zipf(3000, 72)
    with B.Server(n_slots=1, max_queue=1) as srv:
        codes = []
        for _ in range(3):
            try:
                srv.submit(B.MOCHY_REQ_EXACT, *g)
                codes.append(0)
            except B.MochyError as e:
                codes.append(e.code)
        assert codes[0] == 0 and B.E_BUSY in codes[1:]
        with pytest.raises(B.MochyError) as e:
            srv.submit(9, *g)
        assert e.value.code == B.E_INVALID
        with pytest.raises(B.MochyError) as e:
            srv.submit(B.MOCHY_REQ_SAMPLED, *g, samples=0)
        assert e.value.code == B.E_INVALID


def test_large_aplus_requests_run_without_the_line_graph():
    """A MoCHy-A+ request whose line graph would take more than a quarter of
    the budget is served without it: admitted with the smaller reservation,
    and its raw counts, estimates and |wedges| equal the projected call's."""
    g = _zipf(5000, 80)
    est = _estimate(*g)
    with B.Server(n_slots=2, budget=2 * est) as srv:
        t = srv.submit(B.MOCHY_REQ_SAMPLED, *g, samples=4000, seed=9)
        r = srv.poll(t, wait_ms=120000)
        st = srv.stats()
    _check_same(r, _alone(B.MOCHY_REQ_SAMPLED, g, samples=4000, seed=9))
    assert 0 < st["peak_reserved_bytes"] < est
    with B.Context() as c:
        c.load(*g)
        assert r["n_wedges"] == c.project()[0]


def test_large_request_is_not_overtaken_forever():
    """A request too large to start beside the running ones may be overtaken
    by later, smaller requests, but only a bounded number of times: with 60
    small requests queued behind it, it starts before the last of them, and
    every result is still the one the same call gives alone."""
    big, small = _zipf(3000, 81), _zipf(800, 82)
    est_big, est_small = _estimate(*big), _estimate(*small)
    assert est_big > 3 * est_small
    budget = est_big + est_small + est_small // 2     # the big one needs all but one small
    with B.Server(n_slots=4, budget=budget) as srv:
        first = [srv.submit(B.MOCHY_REQ_EXACT, *small) for _ in range(3)]
        t_big = srv.submit(B.MOCHY_REQ_EXACT, *big)
        rest = [srv.submit(B.MOCHY_REQ_EXACT, *small) for _ in range(60)]
        res = {t: srv.poll(t, wait_ms=300000) for t in first + [t_big] + rest}
    assert all(r is not None and r["status"] >= 0 for r in res.values())
    start = {t: r["latency_ms"] - r["service_ms"] for t, r in res.items()}
    # some small request queued behind the big one started after it
    assert max(start[t] for t in rest) > start[t_big]
    _check_same(res[t_big], _alone(B.MOCHY_REQ_EXACT, big))
    ref_small = _alone(B.MOCHY_REQ_EXACT, small)
    for t in first + rest:
        _check_same(res[t], ref_small)
