"""Thin ctypes binding of libmochy (include/mochy.h).

Functions carry the C names and only marshal arguments: numpy arrays in,
numpy arrays out, negative return codes raised as MochyError.  Every step of
the computation runs in the CUDA library; if the library is missing, loading
it fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmochy.so")

N_H, N_3H = 26, 431
MOCHY_A, MOCHY_A_PLUS = 1, 2
OK, W_DEGENERATE_CP = 0, 1
E_INVALID, E_NOMEM, E_CUDA, E_TIMEOUT, E_NOT_PROJECTED, E_UNSUPPORTED, E_BUSY = \
    -1, -2, -3, -4, -5, -6, -7

# every symbol declared in include/mochy.h
EXPORTS = [
    "mochy_config_default", "mochy_create", "mochy_destroy", "mochy_load", "mochy_load_device",
    "mochy_get_hypergraph", "mochy_project", "mochy_line_degrees", "mochy_count_exact",
    "mochy_count_exact_subset", "mochy_count_exact_rows", "mochy_count_sampled", "mochy_randomize", "mochy_profile",
    "mochy_motif_pattern", "mochy_stream", "mochy_device_bytes", "mochy_kernel_launches",
    "mochy_strerror", "mochy_last_error", "mochy_trace", "mochy_trace_read",
    "mochy_count_sampled_noalloc", "mochy_profile_batch", "mochy_server_create",
    "mochy_hyperedge_profile", "mochy_star_node_profile", "mochy_radial_node_profile",
    "mochy_count_kh", "mochy_kh_pattern", "mochy_enumerate", "mochy_count_sampled_onthefly",
    "mochy_tune_dense_threshold",
    "mochy_server_submit", "mochy_server_poll", "mochy_server_stats", "mochy_server_destroy",
]
MOCHY_REQ_EXACT, MOCHY_REQ_SAMPLED, MOCHY_REQ_PROFILE = 1, 2, 3


class MochyError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: code {code}: {msg}")
        self.code = code


class mochy_config(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_int32), ("eps", ctypes.c_double),
                ("hbm_budget_bytes", ctypes.c_int64), ("device", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("exact_kernel", ctypes.c_int32),
                ("dense_threshold", ctypes.c_int32), ("rest_path", ctypes.c_int32)]


class mochy_batch_info(ctypes.Structure):
    _fields_ = [("ms_generate", ctypes.c_double), ("ms_project", ctypes.c_double),
                ("ms_prepare", ctypes.c_double), ("ms_count", ctypes.c_double),
                ("ms_finish", ctypes.c_double), ("n_waves", ctypes.c_int64),
                ("n_units", ctypes.c_int64), ("max_units_per_wave", ctypes.c_int64),
                ("n_edges", ctypes.c_int64), ("n_wedges", ctypes.c_int64),
                ("instances", ctypes.c_int64), ("dense_threshold", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class mochy_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_nodes", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("edge_offsets", ctypes.c_void_p), ("edge_nodes", ctypes.c_void_p),
                ("method", ctypes.c_int32), ("samples", ctypes.c_int64),
                ("n_random", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class mochy_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_wedges", ctypes.c_int64),
                ("counts_h", ctypes.c_int64 * N_H), ("counts_3h", ctypes.c_int64 * N_3H),
                ("est_h", ctypes.c_double * N_H), ("est_3h", ctypes.c_double * N_3H),
                ("sig_h", ctypes.c_double * N_H), ("cp_h", ctypes.c_double * N_H),
                ("sig_3h", ctypes.c_double * N_3H), ("cp_3h", ctypes.c_double * N_3H),
                ("queue_ms", ctypes.c_double), ("service_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("error", ctypes.c_char * 128)]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if isinstance(v, bytes):
                d[name] = v.decode(errors="replace")
            else:
                d[name] = np.ctypeslib.as_array(v).copy() if isinstance(v, ctypes.Array) else v
        return d


class mochy_serving_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "rejected",
                                              "queued", "in_flight", "peak_in_flight",
                                              "budget_bytes", "peak_reserved_bytes")] + \
               [(n, ctypes.c_double) for n in ("p50_ms", "p99_ms", "mean_ms", "max_ms",
                                               "throughput_rps")]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libmochy.so (built by paper_2310_15668_gb300.build); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise OSError(f"libmochy is not built ({path}); run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            lib.mochy_strerror.restype = ctypes.c_char_p
            lib.mochy_strerror.argtypes = [ctypes.c_int]
            lib.mochy_last_error.restype = ctypes.c_char_p
            lib.mochy_last_error.argtypes = []
            lib.mochy_stream.restype = vp
            lib.mochy_stream.argtypes = [vp]
            lib.mochy_device_bytes.restype = i64
            lib.mochy_device_bytes.argtypes = [vp]
            lib.mochy_kernel_launches.restype = i64
            lib.mochy_kernel_launches.argtypes = []
            lib.mochy_config_default.restype = None
            lib.mochy_config_default.argtypes = [ctypes.POINTER(mochy_config)]
            lib.mochy_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(mochy_config)]
            lib.mochy_destroy.argtypes = [vp]
            lib.mochy_load.argtypes = [vp, i64, i64, vp, vp, vp]
            lib.mochy_load_device.argtypes = [vp, i64, i64, vp, vp, vp]
            lib.mochy_get_hypergraph.argtypes = [vp, vp, vp, vp, vp, vp]
            lib.mochy_project.argtypes = [vp, vp, vp]
            lib.mochy_line_degrees.argtypes = [vp, vp]
            lib.mochy_count_exact.argtypes = [vp, vp, vp]
            lib.mochy_count_exact_subset.argtypes = [vp, vp, i64, vp, vp]
            lib.mochy_count_exact_rows.argtypes = [vp, vp, i64, vp, vp]
            lib.mochy_count_sampled.argtypes = [vp, ctypes.c_int, i64, ctypes.c_uint64, vp, vp,
                                                vp, vp]
            lib.mochy_randomize.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.POINTER(vp)]
            lib.mochy_profile.argtypes = [vp, i32, ctypes.c_uint64, vp, vp, vp, vp, vp, vp]
            lib.mochy_motif_pattern.argtypes = [ctypes.c_int, i32, vp]
            lib.mochy_trace.argtypes = [vp, ctypes.c_int]
            lib.mochy_count_sampled_noalloc.argtypes = [vp, ctypes.c_int, i64, ctypes.c_uint64,
                                                        vp, vp, vp, vp]
            lib.mochy_trace_read.argtypes = [vp, ctypes.c_char_p, i64]
            lib.mochy_profile_batch.argtypes = [ctypes.POINTER(mochy_config), i32, vp, vp, vp, vp,
                                                i32, vp, vp, vp, vp, vp, vp, vp, vp,
                                                ctypes.POINTER(mochy_batch_info)]
            lib.mochy_hyperedge_profile.argtypes = [vp, vp, vp]
            lib.mochy_star_node_profile.argtypes = [vp, vp, vp]
            lib.mochy_radial_node_profile.argtypes = [vp, vp, vp]
            lib.mochy_count_kh.argtypes = [vp, i32, vp, vp, vp, i64, vp]
            lib.mochy_kh_pattern.argtypes = [vp, i32, i32, vp]
            lib.mochy_enumerate.argtypes = [vp, i64, vp, vp]
            lib.mochy_tune_dense_threshold.argtypes = [vp, vp, i32, ctypes.c_double,
                                                       ctypes.c_uint64, vp, vp, vp]
            lib.mochy_count_sampled_onthefly.argtypes = [vp, i64, ctypes.c_uint64, i64, vp, vp,
                                                         vp, vp, vp]
            lib.mochy_server_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(mochy_config),
                                                i32, i32]
            lib.mochy_server_submit.argtypes = [vp, ctypes.POINTER(mochy_request),
                                                ctypes.POINTER(i64)]
            lib.mochy_server_poll.argtypes = [vp, i64, ctypes.POINTER(mochy_result), i32]
            lib.mochy_server_stats.argtypes = [vp, ctypes.POINTER(mochy_serving_stats)]
            lib.mochy_server_destroy.argtypes = [vp]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, where: str) -> int:
    if rc < 0:
        lib = load_library()
        raise MochyError(rc, where, lib.mochy_last_error().decode())
    return rc


def mochy_config_default() -> mochy_config:
    cfg = mochy_config()
    load_library().mochy_config_default(ctypes.byref(cfg))
    return cfg


def mochy_create(cfg: mochy_config | None = None) -> int:
    h = ctypes.c_void_p()
    _check(load_library().mochy_create(ctypes.byref(h), None if cfg is None else ctypes.byref(cfg)),
           "mochy_create")
    return h.value


def mochy_destroy(ctx: int) -> None:
    load_library().mochy_destroy(ctx)


def mochy_load(ctx: int, n_nodes: int, offsets: np.ndarray, nodes: np.ndarray) -> int:
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nod = np.ascontiguousarray(nodes, dtype=np.int32)
    dup = np.zeros(1, np.int64)
    _check(load_library().mochy_load(ctx, n_nodes, off.size - 1, _p(off),
                                     _p(nod if nod.size else np.zeros(1, np.int32)), _p(dup)),
           "mochy_load")
    return int(dup[0])


def mochy_load_device(ctx: int, n_nodes: int, n_edges: int, d_offsets: int, d_nodes: int) -> int:
    dup = np.zeros(1, np.int64)
    _check(load_library().mochy_load_device(ctx, n_nodes, n_edges, d_offsets, d_nodes, _p(dup)),
           "mochy_load_device")
    return int(dup[0])


def mochy_get_hypergraph(ctx: int):
    lib = load_library()
    n = np.zeros(3, np.int64)
    _check(lib.mochy_get_hypergraph(ctx, _p(n[0:1]), _p(n[1:2]), _p(n[2:3]), None, None),
           "mochy_get_hypergraph")
    off = np.zeros(int(n[1]) + 1, np.int64)
    nodes = np.zeros(max(int(n[2]), 1), np.int32)
    _check(lib.mochy_get_hypergraph(ctx, None, None, None, _p(off), _p(nodes)),
           "mochy_get_hypergraph")
    return int(n[0]), off, nodes[:int(n[2])]


def mochy_project(ctx: int):
    nw = np.zeros(1, np.int64)
    md = np.zeros(1, np.int32)
    _check(load_library().mochy_project(ctx, _p(nw), _p(md)), "mochy_project")
    return int(nw[0]), int(md[0])


def mochy_line_degrees(ctx: int, n_edges: int) -> np.ndarray:
    d = np.zeros(max(n_edges, 1), np.int64)
    _check(load_library().mochy_line_degrees(ctx, _p(d)), "mochy_line_degrees")
    return d[:n_edges]


def mochy_count_exact(ctx: int):
    h = np.zeros(N_H, np.int64)
    h3 = np.zeros(N_3H, np.int64)
    _check(load_library().mochy_count_exact(ctx, _p(h), _p(h3)), "mochy_count_exact")
    return h, h3


def mochy_count_exact_subset(ctx: int, anchors) -> tuple:
    a = np.ascontiguousarray(anchors, dtype=np.int32)
    h = np.zeros(N_H, np.int64)
    h3 = np.zeros(N_3H, np.int64)
    _check(load_library().mochy_count_exact_subset(ctx, _p(a if a.size else np.zeros(1, np.int32)),
                                                   a.size, _p(h), _p(h3)),
           "mochy_count_exact_subset")
    return h, h3


def mochy_count_exact_rows(ctx: int, rows) -> tuple:
    a = np.ascontiguousarray(rows, dtype=np.int32)
    h = np.zeros(N_H, np.int64)
    h3 = np.zeros(N_3H, np.int64)
    _check(load_library().mochy_count_exact_rows(ctx, _p(a if a.size else np.zeros(1, np.int32)),
                                                 a.size, _p(h), _p(h3)),
           "mochy_count_exact_rows")
    return h, h3


def mochy_count_sampled(ctx: int, method: int, samples: int, seed: int):
    rh = np.zeros(N_H, np.int64)
    r3 = np.zeros(N_3H, np.int64)
    eh = np.zeros(N_H, np.float64)
    e3 = np.zeros(N_3H, np.float64)
    _check(load_library().mochy_count_sampled(ctx, method, samples, ctypes.c_uint64(seed), _p(rh),
                                              _p(r3), _p(eh), _p(e3)), "mochy_count_sampled")
    return rh, r3, eh, e3


def mochy_count_sampled_noalloc(ctx: int, method: int, samples: int, seed: int, d_raw_h: int,
                                d_raw_3h: int, d_est_h: int, d_est_3h: int) -> None:
    """Sampled counts into caller-provided device arrays, with no device
    allocation (for callers that cannot allocate while they run)."""
    _check(load_library().mochy_count_sampled_noalloc(ctx, method, samples, ctypes.c_uint64(seed),
                                                      d_raw_h, d_raw_3h, d_est_h, d_est_3h),
           "mochy_count_sampled_noalloc")


def mochy_randomize(ctx: int, seed: int, copy: int) -> int:
    h = ctypes.c_void_p()
    _check(load_library().mochy_randomize(ctx, ctypes.c_uint64(seed), ctypes.c_uint32(copy),
                                          ctypes.byref(h)), "mochy_randomize")
    return h.value


def mochy_profile(ctx: int, n_random: int, seed: int):
    sig_h = np.zeros(N_H)
    cp_h = np.zeros(N_H)
    sig_3h = np.zeros(N_3H)
    cp_3h = np.zeros(N_3H)
    ch = np.zeros((1 + n_random, N_H), np.int64)
    c3 = np.zeros((1 + n_random, N_3H), np.int64)
    rc = _check(load_library().mochy_profile(ctx, n_random, ctypes.c_uint64(seed), _p(sig_h),
                                             _p(cp_h), _p(sig_3h), _p(cp_3h), _p(ch), _p(c3)),
                "mochy_profile")
    return dict(sig_h=sig_h, cp_h=cp_h, sig_3h=sig_3h, cp_3h=cp_3h, counts_h=ch, counts_3h=c3,
                degenerate=rc == W_DEGENERATE_CP)


def mochy_hyperedge_profile(ctx: int, n_edges: int):
    """Hyperedge profiles of the projected hypergraph: (hp_h [E, 26], hp_3h [E, 431])."""
    hp_h = np.zeros((max(n_edges, 1), N_H), np.int64)
    hp_3h = np.zeros((max(n_edges, 1), N_3H), np.int64)
    _check(load_library().mochy_hyperedge_profile(ctx, _p(hp_h), _p(hp_3h)),
           "mochy_hyperedge_profile")
    return hp_h[:n_edges], hp_3h[:n_edges]


def mochy_star_node_profile(ctx: int, n_nodes: int):
    """Star node profiles of the projected hypergraph: (np_h [N, 26], np_3h [N, 431])."""
    np_h = np.zeros((max(n_nodes, 1), N_H), np.int64)
    np_3h = np.zeros((max(n_nodes, 1), N_3H), np.int64)
    _check(load_library().mochy_star_node_profile(ctx, _p(np_h), _p(np_3h)),
           "mochy_star_node_profile")
    return np_h[:n_nodes], np_3h[:n_nodes]


def mochy_radial_node_profile(ctx: int, n_nodes: int):
    """Radial node profiles of the projected hypergraph: (np_h [N, 26], np_3h [N, 431])."""
    np_h = np.zeros((max(n_nodes, 1), N_H), np.int64)
    np_3h = np.zeros((max(n_nodes, 1), N_3H), np.int64)
    _check(load_library().mochy_radial_node_profile(ctx, _p(np_h), _p(np_3h)),
           "mochy_radial_node_profile")
    return np_h[:n_nodes], np_3h[:n_nodes]


def mochy_count_kh(ctx: int, k: int, thresholds=()):
    """kh-motif counts: (h counts [26], kh counts [X(k)])."""
    thr = np.ascontiguousarray(thresholds, dtype=np.int32)
    n = np.zeros(1, np.int64)
    lib = load_library()
    _check(lib.mochy_count_kh(ctx, k, _p(thr if thr.size else np.zeros(1, np.int32)), None, None,
                              0, _p(n)), "mochy_count_kh")
    h = np.zeros(N_H, np.int64)
    kh = np.zeros(max(int(n[0]), 1), np.int64)
    _check(lib.mochy_count_kh(ctx, k, _p(thr if thr.size else np.zeros(1, np.int32)), _p(h),
                              _p(kh), kh.size, _p(n)), "mochy_count_kh")
    return h, kh[:int(n[0])]


def mochy_count_sampled_onthefly(ctx: int, samples: int, seed: int, budget: int = 0):
    """MoCHy-A+ without the line graph: (raw_h, raw_3h, est_h, est_3h, |wedges|)."""
    rh = np.zeros(N_H, np.int64)
    r3 = np.zeros(N_3H, np.int64)
    eh = np.zeros(N_H, np.float64)
    e3 = np.zeros(N_3H, np.float64)
    nw = np.zeros(1, np.int64)
    _check(load_library().mochy_count_sampled_onthefly(ctx, samples, seed, budget, _p(rh),
                                                        _p(r3), _p(eh), _p(e3), _p(nw)),
           "mochy_count_sampled_onthefly")
    return rh, r3, eh, e3, int(nw[0])


def mochy_tune_dense_threshold(ctx: int, candidates=(), sample_fraction: float = 0.02,
                               seed: int = 1):
    """Measured dense threshold: (best, [(candidate, ms)]); the context
    keeps the best for its following counts."""
    c = np.ascontiguousarray(candidates, dtype=np.int32)
    n = c.size if c.size else 5
    ms = np.zeros(n, np.float64)
    tried = np.zeros(n, np.int32)
    best = np.zeros(1, np.int32)
    _check(load_library().mochy_tune_dense_threshold(
        ctx, _p(c) if c.size else None, int(c.size), float(sample_fraction), seed, _p(best),
        _p(tried), _p(ms)), "mochy_tune_dense_threshold")
    return int(best[0]), list(zip(tried.tolist(), ms.tolist()))


def mochy_kh_pattern(ctx: int, k: int, motif_id: int) -> np.ndarray:
    out = np.zeros(7, np.uint8)
    _check(load_library().mochy_kh_pattern(ctx, k, motif_id, _p(out)), "mochy_kh_pattern")
    return out


def mochy_enumerate(ctx: int, capacity: int):
    """Instances as rows (i, j, k, h id, 3h id), i < j < k, in no particular
    order: (rows [min(n, capacity), 5], n)."""
    out = np.zeros((max(capacity, 1), 5), np.int32)
    n = np.zeros(1, np.int64)
    _check(load_library().mochy_enumerate(ctx, capacity, _p(out), _p(n)), "mochy_enumerate")
    return out[:min(int(n[0]), capacity)], int(n[0])


def mochy_profile_batch(graphs, n_random: int, seeds, cfg: mochy_config | None = None):
    """Profiles of several hypergraphs at once.  graphs: list of
    (n_nodes, offsets, nodes); seeds: one per graph.  Returns
    (sig_h [G,26], cp_h [G,26], sig_3h [G,431], cp_3h [G,431],
    counts_h [G,1+R,26], counts_3h [G,1+R,431], degenerate [G], info dict)."""
    G = len(graphs)
    offs = [np.ascontiguousarray(o, dtype=np.int64) for _, o, _ in graphs]
    nods = [np.ascontiguousarray(v, dtype=np.int32) for _, _, v in graphs]
    nods = [v if v.size else np.zeros(1, np.int32) for v in nods]
    n_nodes = np.array([int(n) for n, _, _ in graphs], np.int64)
    n_edges = np.array([o.size - 1 for o in offs], np.int64)
    po = (ctypes.c_void_p * max(G, 1))(*[o.ctypes.data for o in offs])
    pn = (ctypes.c_void_p * max(G, 1))(*[v.ctypes.data for v in nods])
    sd = np.ascontiguousarray(seeds, dtype=np.uint64)
    if sd.size == 0:
        sd = np.zeros(1, np.uint64)
    sig_h = np.zeros((G, N_H)); cp_h = np.zeros((G, N_H))
    sig_3h = np.zeros((G, N_3H)); cp_3h = np.zeros((G, N_3H))
    ch = np.zeros((G, max(n_random, 0) + 1, N_H), np.int64)
    c3 = np.zeros((G, max(n_random, 0) + 1, N_3H), np.int64)
    deg = np.zeros(max(G, 1), np.int32)
    info = mochy_batch_info()
    _check(load_library().mochy_profile_batch(
        None if cfg is None else ctypes.byref(cfg), G, _p(n_nodes if G else np.zeros(1, np.int64)),
        _p(n_edges if G else np.zeros(1, np.int64)), ctypes.cast(po, ctypes.c_void_p),
        ctypes.cast(pn, ctypes.c_void_p), n_random, _p(sd), _p(sig_h), _p(cp_h), _p(sig_3h),
        _p(cp_3h), _p(ch), _p(c3), _p(deg), ctypes.byref(info)), "mochy_profile_batch")
    return sig_h, cp_h, sig_3h, cp_3h, ch, c3, deg[:G], info.as_dict()


def mochy_motif_pattern(kind: int, motif_id: int) -> np.ndarray:
    out = np.zeros(7, np.uint8)
    _check(load_library().mochy_motif_pattern(kind, motif_id, _p(out)), "mochy_motif_pattern")
    return out


def mochy_stream(ctx: int) -> int:
    return load_library().mochy_stream(ctx) or 0


def mochy_device_bytes(ctx: int) -> int:
    return int(load_library().mochy_device_bytes(ctx))


def mochy_trace(ctx: int, level: int) -> None:
    _check(load_library().mochy_trace(ctx, int(level)), "mochy_trace")


def mochy_trace_read(ctx: int) -> dict:
    import json
    buf = ctypes.create_string_buffer(4096)
    _check(load_library().mochy_trace_read(ctx, buf, 4096), "mochy_trace_read")
    return json.loads(buf.value.decode())


def mochy_kernel_launches() -> int:
    return int(load_library().mochy_kernel_launches())


class Context:
    """Owns one mochy_ctx; `with Context() as c: ...` destroys it on exit."""

    def __init__(self, theta: int = 1, eps: float = 1.0, budget: int = 0, device: int = 0,
                 stream: int | None = None, handle: int | None = None, exact_kernel: int = 0,
                 dense_threshold: int = 0, rest_path: int = 0):
        if handle is not None:
            self.h = handle
        else:
            cfg = mochy_config_default()
            cfg.theta, cfg.eps, cfg.hbm_budget_bytes, cfg.device = theta, eps, budget, device
            cfg.stream = stream
            cfg.exact_kernel, cfg.dense_threshold = exact_kernel, dense_threshold
            cfg.rest_path = rest_path
            self.h = mochy_create(cfg)

    def close(self):
        if self.h:
            mochy_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, n_nodes, offsets, nodes):
        return mochy_load(self.h, n_nodes, offsets, nodes)

    def project(self):
        return mochy_project(self.h)

    def count_exact(self):
        return mochy_count_exact(self.h)

    def count_exact_subset(self, anchors):
        return mochy_count_exact_subset(self.h, anchors)

    def count_exact_rows(self, rows):
        return mochy_count_exact_rows(self.h, rows)

    def count_sampled(self, method, samples, seed):
        return mochy_count_sampled(self.h, method, samples, seed)

    def randomize(self, seed, copy):
        return Context(handle=mochy_randomize(self.h, seed, copy))

    def profile(self, n_random, seed):
        return mochy_profile(self.h, n_random, seed)

    def hyperedge_profile(self):
        _, off, _ = self.hypergraph()
        return mochy_hyperedge_profile(self.h, off.size - 1)

    def star_node_profile(self):
        n_nodes, _, _ = self.hypergraph()
        return mochy_star_node_profile(self.h, n_nodes)

    def radial_node_profile(self):
        n_nodes, _, _ = self.hypergraph()
        return mochy_radial_node_profile(self.h, n_nodes)

    def count_kh(self, k, thresholds=()):
        return mochy_count_kh(self.h, k, thresholds)

    def enumerate(self, capacity):
        return mochy_enumerate(self.h, capacity)

    def count_sampled_onthefly(self, samples, seed, budget=0):
        return mochy_count_sampled_onthefly(self.h, samples, seed, budget)

    def hypergraph(self):
        return mochy_get_hypergraph(self.h)

    def line_degrees(self):
        n_nodes, off, _ = self.hypergraph()
        return mochy_line_degrees(self.h, off.size - 1)

    @property
    def stream(self):
        return mochy_stream(self.h)


class Server:
    """A mochy_server: continuous batching of count / sampled / profile
    requests over n_slots workers (each with its own context and stream)."""

    def __init__(self, n_slots: int = 4, max_queue: int = 1 << 16, budget: int = 0,
                 device: int = 0, dense_threshold: int = 0):
        cfg = mochy_config_default()
        cfg.hbm_budget_bytes, cfg.device, cfg.dense_threshold = budget, device, dense_threshold
        h = ctypes.c_void_p()
        _check(load_library().mochy_server_create(ctypes.byref(h), ctypes.byref(cfg), n_slots,
                                                  max_queue), "mochy_server_create")
        self.h = h.value

    def submit(self, kind: int, n_nodes: int, offsets, nodes, method: int = MOCHY_A_PLUS,
               samples: int = 0, n_random: int = 0, seed: int = 0) -> int:
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        nod = np.ascontiguousarray(nodes, dtype=np.int32)
        req = mochy_request(kind, n_nodes, off.size - 1, off.ctypes.data,
                            nod.ctypes.data if nod.size else None, method, samples, n_random,
                            seed)
        t = ctypes.c_int64()
        _check(load_library().mochy_server_submit(self.h, ctypes.byref(req), ctypes.byref(t)),
               "mochy_server_submit")
        return t.value

    def poll(self, ticket: int, wait_ms: int = 0):
        res = mochy_result()
        rc = _check(load_library().mochy_server_poll(self.h, ticket, ctypes.byref(res), wait_ms),
                    "mochy_server_poll")
        return res.as_dict() if rc == 1 else None

    def stats(self) -> dict:
        st = mochy_serving_stats()
        _check(load_library().mochy_server_stats(self.h, ctypes.byref(st)), "mochy_server_stats")
        return st.as_dict()

    def close(self):
        if self.h:
            load_library().mochy_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
