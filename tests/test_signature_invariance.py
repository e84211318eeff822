"""The grouping rule behind the dense-triangle kernel's signature slots.

For theta = 1 the kernel sums the popcounted closed-instance bins of all
hyperwedges (a, b) of a row that share the signature (min(x, 4),
min(A - x, 4), min(B - x, 5), min(B, 5)) and classifies them once, with one
representative hyperwedge.  That is exact only if every bin's motif code and
its three "as if open" codes (Lemma "motif:time" regions, states 0 / 1 / 2+)
are the same for every (A, x, B) with the same signature; this checks it
exhaustively for |e| up to 40.
"""


def _state(r):
    assert r >= 0
    return 0 if r == 0 else (1 if r <= 1 else 2)


def _regions(A, B, C, x, y, z, t):
    return tuple(_state(r) for r in (A - x - z + t, B - x - y + t, C - y - z + t, x - t, y - t,
                                     z - t, t))


# (xa, xb, xt, smallest effective size, number of size bins)
_POP = [(0, 0, 1, 1, 4), (0, 1, 1, 2, 4), (1, 0, 1, 2, 4), (1, 1, 0, 2, 3), (0, 2, 1, 3, 4),
        (1, 1, 1, 3, 4), (0, 0, 2, 2, 5)]
_BINS = [(xa, xb, xt, c0 + k) for xa, xb, xt, c0, n in _POP for k in range(n)]


def _codes(A, B, x):
    out = []
    for xa, xb, xt, C in _BINS:
        y, z, t = xb + xt, xa + xt, xt
        if A - x - z + t < 0 or B - x - y + t < 0 or C - y - z + t < 0 or x - t < 0:
            out.append(None)
            continue
        out.append((_regions(A, B, C, x, y, z, t),
                    _regions(A, B, C, x, 0, z, 0) if x + z <= A else None,
                    _regions(B, A, C, x, 0, y, 0) if x + y <= B else None,
                    _regions(C, A, B, z, 0, y, 0) if z + y <= C else None))
    return out


def test_codes_depend_only_on_the_signature():
    assert len(_BINS) == 28
    for A in range(1, 41):
        seen = {}
        for x in range(1, A + 1):
            for B in range(x, 41):
                key = (min(x, 4), min(A - x, 4), min(B - x, 5), min(B, 5))
                codes = _codes(A, B, x)
                assert seen.setdefault(key, codes) == codes, (A, x, B)


def test_a_coarser_signature_would_not_be_exact():
    # dropping min(A - x, 4) merges hyperwedges whose closed codes differ
    A = 5
    assert _codes(A, 9, 4) != _codes(A, 9, 5)
