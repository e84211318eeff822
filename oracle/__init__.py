"""Reference oracle for MoCHy motif counting (TEST INFRASTRUCTURE ONLY).

A plain, slow C++ restatement of the paper's algorithms
(``mochy_oracle.cpp``), loaded with ctypes; one thread, except the anchor
loop of ``count_exact_ranked`` and ``line_degrees`` (host threads, the
paper's parallel scheme).  Only the test suite, the smoke
check and the bench's CPU-baseline leg may import this package; the CUDA
library never does, and this package never imports the library.

Functions whose parity is pinned by tests/test_oracle_*.py:
  tables, count_kh           motif tables and the kh-motif chain
  philox                     Philox4x32-10 known answers
  dedupe, project            load and line-graph construction
  count_exact, count_exact_subset, count_exact_ranked, line_degrees
  count_sampled              MoCHy-A / MoCHy-A+
  randomize, profile         Chung-Lu null model, significance, CP
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mochy_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

N_H, N_3H = 26, 431
A, A_PLUS = 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with the host compiler (plain -O2; OpenMP for the
    anchor loops when the compiler has it, else one thread)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC]
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def host_threads() -> int:
    """Host cores this process may use."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.orc_count_kh.restype = ctypes.c_int64
            _lib.orc_count_kh.argtypes = [ctypes.c_int]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(offsets, nodes):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nod = np.ascontiguousarray(nodes, dtype=np.int32)
    if nod.size == 0:
        nod = np.zeros(1, np.int32)
    return off, nod


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def tables():
    """Motif tables: dict of lut_h[128], lut_3h[2187], patterns, t_to_h, open."""
    lib = _load()
    lut_h = np.zeros(128, np.int32)
    lut_3h = np.zeros(2187, np.int32)
    hp = np.zeros((N_H, 7), np.uint8)
    tp = np.zeros((N_3H, 7), np.uint8)
    t2h = np.zeros(N_3H, np.int32)
    hopen = np.zeros(N_H, np.uint8)
    chain = np.zeros(8, np.int64)
    _check(lib.orc_tables(_p(lut_h), _p(lut_3h), _p(hp), _p(tp), _p(t2h), _p(hopen),
                          _p(chain)), "tables")
    return dict(lut_h=lut_h, lut_3h=lut_3h, h_pattern=hp, t_pattern=tp, t_to_h=t2h,
                h_open=hopen, chain=chain)


def count_kh(k: int) -> int:
    return int(_load().orc_count_kh(int(k)))


def philox(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    _check(_load().orc_philox(_p(c), _p(k), _p(o)), "philox")
    return o


def dedupe(offsets, nodes):
    off, nod = _csr(offsets, nodes)
    e = off.size - 1
    out_off = np.zeros(e + 1, np.int64)
    out_nodes = np.zeros(max(nod.size, 1), np.int32)
    n_out = np.zeros(1, np.int64)
    n_dup = np.zeros(1, np.int64)
    _check(_load().orc_dedupe(ctypes.c_int64(e), _p(off), _p(nod), _p(out_off),
                              _p(out_nodes), _p(n_out), _p(n_dup)), "dedupe")
    n = int(n_out[0])
    return out_off[:n + 1].copy(), out_nodes[:out_off[n]].copy(), int(n_dup[0])


def project(offsets, nodes):
    """(|wedges|, max line-graph degree, degrees[E])."""
    off, nod = _csr(offsets, nodes)
    e = off.size - 1
    nw = np.zeros(1, np.int64)
    md = np.zeros(1, np.int64)
    deg = np.zeros(max(e, 1), np.int64)
    _check(_load().orc_project(ctypes.c_int64(e), _p(off), _p(nod), _p(nw), _p(md),
                               _p(deg)), "project")
    return int(nw[0]), int(md[0]), deg[:e]


def count_exact(offsets, nodes, theta: int = 1):
    off, nod = _csr(offsets, nodes)
    h = np.zeros(N_H, np.int64)
    h3 = np.zeros(N_3H, np.int64)
    _check(_load().orc_count_exact(ctypes.c_int64(off.size - 1), _p(off), _p(nod),
                                   ctypes.c_int32(theta), _p(h), _p(h3)), "count_exact")
    return h, h3


def hyperedge_profile(offsets, nodes, theta: int = 1):
    """Hyperedge profiles (Section 3.1, "Hyperedge Profile (HP)"): row e
    counts the instances of each h-motif / 3h-motif that include hyperedge e
    (ids after duplicate removal).  Returns (hp_h [E, 26], hp_3h [E, 431])."""
    off, nod = _csr(offsets, nodes)
    e_kept = dedupe(off, nod)[0].size - 1
    hp_h = np.zeros((max(e_kept, 1), N_H), np.int64)
    hp_3h = np.zeros((max(e_kept, 1), N_3H), np.int64)
    _check(_load().orc_hyperedge_profile(ctypes.c_int64(off.size - 1), _p(off), _p(nod),
                                         ctypes.c_int32(theta), _p(hp_h), _p(hp_3h)),
           "hyperedge_profile")
    return hp_h[:e_kept], hp_3h[:e_kept]


def star_node_profile(n_nodes: int, offsets, nodes, theta: int = 1):
    """Star node profiles (Section 3.1, "Node Profile (NP)", star
    ego-networks): row v counts the instances of each h-motif / 3h-motif
    among the hyperedges that contain v.  Returns (np_h [N, 26], np_3h [N, 431])."""
    off, nod = _csr(offsets, nodes)
    np_h = np.zeros((max(n_nodes, 1), N_H), np.int64)
    np_3h = np.zeros((max(n_nodes, 1), N_3H), np.int64)
    _check(_load().orc_star_node_profile(ctypes.c_int64(n_nodes), ctypes.c_int64(off.size - 1),
                                         _p(off), _p(nod), ctypes.c_int32(theta), _p(np_h),
                                         _p(np_3h)), "star_node_profile")
    return np_h[:n_nodes], np_3h[:n_nodes]


def count_exact_subset(offsets, nodes, anchors, theta: int = 1):
    off, nod = _csr(offsets, nodes)
    anc = np.ascontiguousarray(anchors, dtype=np.int32)
    h = np.zeros(N_H, np.int64)
    h3 = np.zeros(N_3H, np.int64)
    _check(_load().orc_count_exact_subset(
        ctypes.c_int64(off.size - 1), _p(off), _p(nod), ctypes.c_int32(theta),
        _p(anc if anc.size else np.zeros(1, np.int32)), ctypes.c_int64(anc.size),
        _p(h), _p(h3)), "count_exact_subset")
    return h, h3


def count_exact_ranked(offsets, nodes, anchors, rank=None, theta: int = 1,
                       threads: int = 1):
    """MoCHy-E restricted to the outer-loop iterations of ``anchors`` with the
    hyperedges compared by ``rank`` (int64 per hyperedge after duplicate
    removal; ``None`` compares ids, as Algorithm "exact_motif_counting"
    does): open instances centred at an anchor plus closed instances whose
    lowest-ranked member is an anchor.  ``threads`` host threads (0 = all)."""
    off, nod = _csr(offsets, nodes)
    anc = np.ascontiguousarray(anchors, dtype=np.int32)
    rk = None if rank is None else np.ascontiguousarray(rank, dtype=np.int64)
    h = np.zeros(N_H, np.int64)
    h3 = np.zeros(N_3H, np.int64)
    nt = host_threads() if threads == 0 else int(threads)
    _check(_load().orc_count_exact_ranked(
        ctypes.c_int64(off.size - 1), _p(off), _p(nod), ctypes.c_int32(theta),
        _p(anc if anc.size else np.zeros(1, np.int32)), ctypes.c_int64(anc.size),
        None if rk is None else _p(rk), ctypes.c_int32(nt), _p(h), _p(h3)),
        "count_exact_ranked")
    return h, h3


def count_exact_threads(offsets, nodes, theta: int = 1, threads: int = 0):
    """The full MoCHy-E count with every hyperedge an anchor, on ``threads``
    host threads (0 = all), neighbourhoods computed on the fly."""
    n_kept = dedupe(offsets, nodes)[0].size - 1
    return count_exact_ranked(offsets, nodes, np.arange(n_kept, dtype=np.int32), None,
                              theta, threads)


def line_degrees(offsets, nodes, threads: int = 0):
    """|N_e| of every hyperedge (after duplicate removal), from the incidence
    lists, without building the line graph."""
    off, nod = _csr(offsets, nodes)
    n_kept = dedupe(off, nod)[0].size - 1
    deg = np.zeros(max(n_kept, 1), np.int64)
    nt = host_threads() if threads == 0 else int(threads)
    _check(_load().orc_line_degrees(ctypes.c_int64(off.size - 1), _p(off), _p(nod),
                                    ctypes.c_int32(nt), _p(deg)), "line_degrees")
    return deg[:n_kept]


def count_sampled(offsets, nodes, method: int, samples: int, seed: int, theta: int = 1):
    off, nod = _csr(offsets, nodes)
    rh = np.zeros(N_H, np.int64)
    r3 = np.zeros(N_3H, np.int64)
    eh = np.zeros(N_H, np.float64)
    e3 = np.zeros(N_3H, np.float64)
    _check(_load().orc_count_sampled(
        ctypes.c_int64(off.size - 1), _p(off), _p(nod), ctypes.c_int32(theta),
        ctypes.c_int(method), ctypes.c_int64(samples), ctypes.c_uint64(seed),
        _p(rh), _p(r3), _p(eh), _p(e3)), "count_sampled")
    return rh, r3, eh, e3


def count_all_anchors(offsets, nodes, method: int, theta: int = 1):
    """Sampling bodies run once per hyperedge (A) or per hyperwedge (A+)."""
    off, nod = _csr(offsets, nodes)
    rh = np.zeros(N_H, np.int64)
    r3 = np.zeros(N_3H, np.int64)
    _check(_load().orc_count_all_anchors(ctypes.c_int64(off.size - 1), _p(off), _p(nod),
                                         ctypes.c_int32(theta), ctypes.c_int(method),
                                         _p(rh), _p(r3)), "count_all_anchors")
    return rh, r3


def randomize(n_nodes: int, offsets, nodes, seed: int, copy: int):
    off, nod = _csr(offsets, nodes)
    e = off.size - 1
    out_off = np.zeros(e + 1, np.int64)
    out_nodes = np.zeros(max(nod.size, 1), np.int32)
    n_out = np.zeros(1, np.int64)
    _check(_load().orc_randomize(ctypes.c_int64(n_nodes), ctypes.c_int64(e), _p(off),
                                 _p(nod), ctypes.c_uint64(seed), ctypes.c_uint32(copy),
                                 _p(out_off), _p(out_nodes), _p(n_out)), "randomize")
    n = int(n_out[0])
    return out_off[:n + 1].copy(), out_nodes[:out_off[n]].copy()


def profile(n_nodes: int, offsets, nodes, n_random: int, seed: int, theta: int = 1,
            eps: float = 1.0):
    """Significance and CP; also the per-graph counts (row 0 = input)."""
    off, nod = _csr(offsets, nodes)
    sig_h = np.zeros(N_H)
    cp_h = np.zeros(N_H)
    sig_3h = np.zeros(N_3H)
    cp_3h = np.zeros(N_3H)
    ch = np.zeros((1 + n_random, N_H), np.int64)
    c3 = np.zeros((1 + n_random, N_3H), np.int64)
    deg = np.zeros(2, np.int32)
    _check(_load().orc_profile(
        ctypes.c_int64(n_nodes), ctypes.c_int64(off.size - 1), _p(off), _p(nod),
        ctypes.c_int32(theta), ctypes.c_int32(n_random), ctypes.c_uint64(seed),
        ctypes.c_double(eps), _p(sig_h), _p(cp_h), _p(sig_3h), _p(cp_3h), _p(ch),
        _p(c3), _p(deg)), "profile")
    return dict(sig_h=sig_h, cp_h=cp_h, sig_3h=sig_3h, cp_3h=cp_3h, counts_h=ch,
                counts_3h=c3, degenerate=deg)


def kh_tables(k: int):
    """kh-motif tables for k states: dict of lut[k^7] (code = sum_p state_p
    k^p -> id, 0 none), pattern [X(k), 7], to_h [X(k)]."""
    lib = _load()
    lib.orc_kh_tables.restype = ctypes.c_int64
    lut = np.zeros(k ** 7, np.int32)
    n = int(lib.orc_kh_tables(ctypes.c_int(k), _p(lut), None, None, ctypes.c_int64(0)))
    if n < 0:
        raise ValueError(f"oracle kh_tables failed for k={k}")
    pat = np.zeros((n, 7), np.uint8)
    to_h = np.zeros(n, np.int32)
    lib.orc_kh_tables(ctypes.c_int(k), _p(lut), _p(pat), _p(to_h), ctypes.c_int64(n))
    return dict(lut=lut, pattern=pat, to_h=to_h)


def count_exact_kh(offsets, nodes, k: int, thresholds):
    """Exact kh-motif counts (k states, k - 2 ascending thresholds):
    returns (h counts [26], kh counts [X(k)])."""
    off, nod = _csr(offsets, nodes)
    thr = np.ascontiguousarray(thresholds, dtype=np.int32)
    if thr.size != k - 2:
        raise ValueError("k - 2 thresholds are needed")
    n = kh_tables(k)["to_h"].size
    h = np.zeros(N_H, np.int64)
    kh = np.zeros(n, np.int64)
    _check(_load().orc_count_exact_kh(ctypes.c_int64(off.size - 1), _p(off), _p(nod),
                                      ctypes.c_int32(k),
                                      _p(thr if thr.size else np.zeros(1, np.int32)),
                                      _p(h), _p(kh)), "count_exact_kh")
    return h, kh


def radial_node_profile(n_nodes: int, offsets, nodes, theta: int = 1):
    """Radial node profiles (Section 3.1, "Node Profile (NP)", radial
    ego-networks): row v counts the instances of each h-motif / 3h-motif
    among the hyperedges contained in the union of the hyperedges that hold
    v.  Returns (np_h [N, 26], np_3h [N, 431])."""
    off, nod = _csr(offsets, nodes)
    np_h = np.zeros((max(n_nodes, 1), N_H), np.int64)
    np_3h = np.zeros((max(n_nodes, 1), N_3H), np.int64)
    _check(_load().orc_radial_node_profile(ctypes.c_int64(n_nodes), ctypes.c_int64(off.size - 1),
                                           _p(off), _p(nod), ctypes.c_int32(theta), _p(np_h),
                                           _p(np_3h)), "radial_node_profile")
    return np_h[:n_nodes], np_3h[:n_nodes]


def enumerate_instances(offsets, nodes, theta: int = 1, cap: int | None = None):
    """Algorithm "alg:enum": every instance as a row (i, j, k, h id, 3h id),
    ids ascending within the row, in the order the algorithm meets them."""
    off, nod = _csr(offsets, nodes)
    n_out = np.zeros(1, np.int64)
    if cap is None:
        h, _ = count_exact(off, nod, theta)
        cap = int(h.sum())
    out = np.zeros((max(cap, 1), 5), np.int32)
    _check(_load().orc_enumerate(ctypes.c_int64(off.size - 1), _p(off), _p(nod),
                                 ctypes.c_int32(theta), ctypes.c_int64(cap), _p(out),
                                 _p(n_out)), "enumerate")
    n = int(n_out[0])
    return out[:min(n, cap)].copy(), n


def significance_cp(M, sum_rand, n_random: int, eps: float = 1.0):
    """Eq. "significance" and Eq. "cp" from the input's counts and the counts
    summed over n_random copies: (significances, CP, degenerate)."""
    m = np.ascontiguousarray(M, dtype=np.int64)
    s = np.ascontiguousarray(sum_rand, dtype=np.int64)
    sig = np.zeros(m.size)
    cp = np.zeros(m.size)
    deg = np.zeros(1, np.int32)
    _check(_load().orc_significance_cp(_p(m), _p(s), ctypes.c_int32(n_random),
                                       ctypes.c_int32(m.size), ctypes.c_double(eps), _p(sig),
                                       _p(cp), _p(deg)), "significance_cp")
    return sig, cp, bool(deg[0])


def count_aplus_onthefly(offsets, nodes, method: int, samples: int, seed: int, budget: int,
                         theta: int = 1):
    """MoCHy-A+ without the line graph: method 1 = basic (Algorithm
    "alg_memdeg"), 2 = advanced (Algorithm "alg_memdeg_adv"), memo budget in
    neighbour entries.  Returns (raw_h, raw_3h, est_h, est_3h, stats) with
    stats = (getNeighbors calls, evictions, |wedges|)."""
    off, nod = _csr(offsets, nodes)
    rh = np.zeros(N_H, np.int64)
    r3 = np.zeros(N_3H, np.int64)
    eh = np.zeros(N_H, np.float64)
    e3 = np.zeros(N_3H, np.float64)
    st = np.zeros(3, np.int64)
    _check(_load().orc_count_aplus_onthefly(
        ctypes.c_int64(off.size - 1), _p(off), _p(nod), ctypes.c_int32(theta), ctypes.c_int(method),
        ctypes.c_int64(samples), ctypes.c_uint64(seed), ctypes.c_int64(budget), _p(rh), _p(r3),
        _p(eh), _p(e3), _p(st)), "count_aplus_onthefly")
    return rh, r3, eh, e3, st


def count_split_rows(offsets, nodes, rows, rank=None, theta: int = 1, threads: int = 1):
    """Per-row shares of the exact count when open instances are counted per
    centre from all neighbour pairs: for each row r, every pair of its
    neighbours classified as if open at r, plus, for each closed instance
    whose lowest-ranked member is r, its motif minus its three as-if-open
    terms.  Summed over all rows this is the exact count.  (h [26], 3h [431]),
    entries may be negative."""
    off, nod = _csr(offsets, nodes)
    rw = np.ascontiguousarray(rows, dtype=np.int32)
    rk = None if rank is None else np.ascontiguousarray(rank, dtype=np.int64)
    h = np.zeros(N_H, np.int64)
    h3 = np.zeros(N_3H, np.int64)
    nt = host_threads() if threads == 0 else int(threads)
    _check(_load().orc_count_split_rows(
        ctypes.c_int64(off.size - 1), _p(off), _p(nod), ctypes.c_int32(theta),
        _p(rw if rw.size else np.zeros(1, np.int32)), ctypes.c_int64(rw.size),
        None if rk is None else _p(rk), ctypes.c_int32(nt), _p(h), _p(h3)), "count_split_rows")
    return h, h3
