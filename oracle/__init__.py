"""CPU oracle for sampled betweenness centrality -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. The product path (``paper_1608_04472_gb300``) never
does, and this package never imports the product path.

The arithmetic lives in ``bc_oracle.c`` (plain single-threaded C, compiled with
``-ffp-contract=off`` so every double operation rounds once). This module only
marshals numpy arrays through ctypes. Function-by-function citations of the
paper are in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bc_oracle.c")
_LIB = os.path.join(_HERE, "_bc_oracle.so")
_lib = None

STOPPED = 0
CAPPED = 1
SIGMA_OVERFLOW = 1

_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32, _i64, _u64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double


def build(force: bool = False) -> str:
    """Compile bc_oracle.c into _bc_oracle.so (in-tree) and return its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    sig = {
        "orc_philox4x64_10": (None, [_u64p, _u64p, _u64p]),
        "orc_draw_source": (_i32, [_u64, _u64, _u64, _i32]),
        "orc_draw_pair": (None, [_u64, _u64, _u64, _i32, _i32p, _i32p]),
        "orc_exact_sum": (_f64, [_f64p, _i64]),
        "orc_bfs": (ctypes.c_int, [_i32, _i32p, _i32p, _i32, _i32p, _u64p, _i32p, _i32p]),
        "orc_source_dependencies": (ctypes.c_int, [_i32, _i32p, _i32p, _i32, _f64p, _i32p, _u64p]),
        "orc_exact_bc": (ctypes.c_int, [_i32, _i32p, _i32p, _f64p]),
        "orc_uniform_sources": (ctypes.c_int, [_i32, _i32p, _i32p, _i64, _u64, _u64, _f64p]),
        "orc_adaptive_sources": (ctypes.c_int, [_i32, _i32p, _i32p, _i32, _i32p, _f64, _i64, _u64,
                                                _u64, _f64p, _i64p, _f64p, _i32p]),
        "orc_adaptive_pairs": (ctypes.c_int, [_i32, _i32p, _i32p, _i32, _i32p, _f64, _i64, _u64,
                                              _u64, _f64, _f64p, _i64p, _f64p, _i32p]),
        "orc_pair_value": (_f64, [_i32, _i32, _i32, _i32p, _u64p, _i32, _u64]),
        "orc_pair_sequence": (ctypes.c_int, [_i32, _i32p, _i32p, _i32, _u64, _u64, _i64, _i64,
                                             _f64p, _i32p, _i32p]),
        "orc_source_dependencies_xf": (ctypes.c_int, [_i32, _i32p, _i32p, _i32, _f64p, _i32p,
                                                      _f64p, _i64p]),
        "orc_xf_add_pair": (None, [_f64, _i64, _f64, _i64, _f64p, _i64p]),
        "orc_pair_value_of": (_f64, [_i32, _i32p, _i32p, _i32, _i32, _i32]),
        "orc_source_dependencies_w": (ctypes.c_int, [_i32, _i32p, _i32p, _u32p, _i32, _f64p, _i64p, _u64p,
                                                     _f64p, _i64p]),
        "orc_exact_bc_w": (ctypes.c_int, [_i32, _i32p, _i32p, _u32p, _f64p]),
        "orc_uniform_sources_w": (ctypes.c_int, [_i32, _i32p, _i32p, _u32p, _i64, _u64, _u64, _f64p]),
        "orc_adaptive_sources_w": (ctypes.c_int, [_i32, _i32p, _i32p, _u32p, _i32, _i32p, _f64, _i64, _u64,
                                                  _u64, _f64p, _i64p, _f64p, _i32p]),
        "orc_accs_new": (ctypes.c_void_p, [_i32]),
        "orc_accs_add_rows": (None, [ctypes.c_void_p, _i32, _i32, _i32, _f64p, _i64]),
        "orc_accs_uniform_est": (None, [ctypes.c_void_p, _i32, _i64, _f64p]),
        "orc_accs_free": (None, [ctypes.c_void_p]),
        "orc_pair_sequence_multi": (ctypes.c_int, [_i32, _i32p, _i32p, _i32, _i32p, _u64, _u64, _i64, _i64,
                                                   _f64p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, np.int32)
    return rp.shape[0] - 1, rp, col


def _check(rc):
    if rc < 0:
        raise ValueError(f"oracle call failed with code {rc}")
    return rc


def philox4x64_10(counter, key):
    """Philox4x64-10 block for a 4-word counter and 2-word key (ints)."""
    c = np.array(counter, dtype=np.uint64)
    k = np.array(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    _load().orc_philox4x64_10(_p(c, _u64p), _p(k, _u64p), _p(out, _u64p))
    return [int(x) for x in out]


def draw_source(seed: int, qid: int, i: int, n: int) -> int:
    return int(_load().orc_draw_source(seed, qid, i, n))


def draw_pair(seed: int, qid: int, i: int, n: int):
    u, t = _i32(), _i32()
    _load().orc_draw_pair(seed, qid, i, n, ctypes.byref(u), ctypes.byref(t))
    return int(u.value), int(t.value)


def exact_sum(values) -> float:
    """Exact sum of non-negative doubles, rounded once to nearest-even."""
    x = np.ascontiguousarray(values, dtype=np.float64)
    if x.size == 0:
        return 0.0
    return float(_load().orc_exact_sum(_p(x, _f64p), x.size))


def bfs(g, s: int):
    """(dist int32[n] with -1 = unreachable, sigma uint64[n], order, overflow flag)."""
    n, rp, col = _csr(g)
    dist = np.empty(n, np.int32)
    sigma = np.empty(n, np.uint64)
    order = np.empty(n, np.int32)
    nr = _i32()
    rc = _check(_load().orc_bfs(n, _p(rp, _i32p), _p(col, _i32p), s, _p(dist, _i32p),
                                _p(sigma, _u64p), _p(order, _i32p), ctypes.byref(nr)))
    return dist, sigma, order[:nr.value], rc == SIGMA_OVERFLOW


def dependencies(g, s: int):
    """(delta float64[n], dist, sigma, overflow) for source s (Theorem 1). When
    overflow is True some count exceeded 2^64-1: delta comes from the extended
    form and sigma holds wrapped counts."""
    n, rp, col = _csr(g)
    delta = np.empty(n, np.float64)
    dist = np.empty(n, np.int32)
    sigma = np.empty(n, np.uint64)
    rc = _check(_load().orc_source_dependencies(n, _p(rp, _i32p), _p(col, _i32p), s,
                                                _p(delta, _f64p), _p(dist, _i32p),
                                                _p(sigma, _u64p)))
    return delta, dist, sigma, rc == SIGMA_OVERFLOW


def dependencies_xf(g, s: int):
    """The per-source step entirely in the extended form (unbounded exponent):
    (delta float64[n], dist int32[n], sigma mantissa float64[n] in [1,2) or 0,
    sigma exponent int64[n]); sigma_sv = mantissa * 2**exponent."""
    n, rp, col = _csr(g)
    delta = np.empty(n, np.float64)
    dist = np.empty(n, np.int32)
    sm = np.empty(n, np.float64)
    se = np.empty(n, np.int64)
    _check(_load().orc_source_dependencies_xf(n, _p(rp, _i32p), _p(col, _i32p), s,
                                              _p(delta, _f64p), _p(dist, _i32p), _p(sm, _f64p),
                                              _p(se, _i64p)))
    return delta, dist, sm, se


def xf_add(m1: float, e1: int, m2: float, e2: int):
    """(m1 2^e1) + (m2 2^e2) rounded once in the extended form -> (m, e)."""
    m, e = _f64(), _i64()
    _load().orc_xf_add_pair(m1, e1, m2, e2, ctypes.byref(m), ctypes.byref(e))
    return float(m.value), int(e.value)


def exact_bc(g) -> np.ndarray:
    """Exact BC over ordered pairs (Eq. 4) for every vertex."""
    n, rp, col = _csr(g)
    bc = np.empty(n, np.float64)
    _check(_load().orc_exact_bc(n, _p(rp, _i32p), _p(col, _i32p), _p(bc, _f64p)))
    return bc


def uniform_sources(g, k: int, seed: int, qid: int) -> np.ndarray:
    n, rp, col = _csr(g)
    est = np.empty(n, np.float64)
    _check(_load().orc_uniform_sources(n, _p(rp, _i32p), _p(col, _i32p), k, seed, qid,
                                       _p(est, _f64p)))
    return est


def adaptive_sources(g, targets, c: float, cap: int, seed: int, qid: int):
    """Bader's adaptive source sampling. Returns dict(est, k, S, status)."""
    n, rp, col = _csr(g)
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    T = tg.size
    est = np.empty(T, np.float64)
    k = np.empty(T, np.int64)
    S = np.empty(T, np.float64)
    st = np.empty(T, np.int32)
    tgp = tg if T else np.zeros(1, np.int32)
    _check(_load().orc_adaptive_sources(n, _p(rp, _i32p), _p(col, _i32p), T, _p(tgp, _i32p),
                                        c, cap, seed, qid, _p(est, _f64p), _p(k, _i64p),
                                        _p(S, _f64p), _p(st, _i32p)))
    return dict(est=est, k=k, S=S, status=st)


def adaptive_pairs(g, targets, c: float, cap: int, seed: int, qid: int,
                   threshold_scale: float = 1.0):
    """Algorithm 1 (adaptive pair sampling). Returns dict(est, k, S, status)."""
    n, rp, col = _csr(g)
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    T = tg.size
    est = np.empty(T, np.float64)
    k = np.empty(T, np.int64)
    S = np.empty(T, np.float64)
    st = np.empty(T, np.int32)
    tgp = tg if T else np.zeros(1, np.int32)
    _check(_load().orc_adaptive_pairs(n, _p(rp, _i32p), _p(col, _i32p), T, _p(tgp, _i32p),
                                      c, cap, seed, qid, threshold_scale, _p(est, _f64p),
                                      _p(k, _i64p), _p(S, _f64p), _p(st, _i32p)))
    return dict(est=est, k=k, S=S, status=st)


def pair_value(v: int, s: int, t: int, dist_v, sigma_v, d_st: int, sigma_st: int) -> float:
    """sigma_st(v)/sigma_st from a BFS at v (dist_v, sigma_v) and d(s,t), sigma_st."""
    dv = np.ascontiguousarray(dist_v, dtype=np.int32)
    sv = np.ascontiguousarray(sigma_v, dtype=np.uint64)
    return float(_load().orc_pair_value(v, s, t, _p(dv, _i32p), _p(sv, _u64p), d_st, sigma_st))


def pair_value_of(g, v: int, s: int, t: int) -> float:
    """sigma_st(v)/sigma_st for one ordered pair, each count in the form the
    estimator uses (exact uint64, or extended when it overflows)."""
    n, rp, col = _csr(g)
    return float(_load().orc_pair_value_of(n, _p(rp, _i32p), _p(col, _i32p), v, s, t))


def pair_sequence(g, v: int, seed: int, qid: int, i0: int, count: int):
    """Per-draw pair dependencies y_i(v) for draws i0..i0+count-1; returns (y, s, t)."""
    n, rp, col = _csr(g)
    y = np.empty(count, np.float64)
    s = np.empty(count, np.int32)
    t = np.empty(count, np.int32)
    _check(_load().orc_pair_sequence(n, _p(rp, _i32p), _p(col, _i32p), v, seed, qid, i0, count,
                                     _p(y, _f64p), _p(s, _i32p), _p(t, _i32p)))
    return y, s, t


# ---- weighted graphs: positive integer lengths w[j] of CSR entry j (Sec. 3, R19) ----

def _wts(g, w):
    w = np.ascontiguousarray(w, dtype=np.uint32)
    if w.shape[0] != np.asarray(g.col).shape[0]:
        raise ValueError("one length per CSR entry")
    return w if w.size else np.ones(1, np.uint32)


def dependencies_w(g, w, s: int):
    """One source on a weighted graph: (delta, dist int64, sigma u64, overflow,
    sigma mantissa, sigma exponent). With overflow the sample is in the
    extended form and sigma holds UINT64_MAX at reached vertices."""
    n, rp, col = _csr(g)
    wt = _wts(g, w)
    delta = np.empty(n, np.float64)
    dist = np.empty(n, np.int64)
    sig = np.empty(n, np.uint64)
    sm = np.empty(n, np.float64)
    se = np.empty(n, np.int64)
    rc = _check(_load().orc_source_dependencies_w(n, _p(rp, _i32p), _p(col, _i32p), _p(wt, _u32p), s,
                                                  _p(delta, _f64p), _p(dist, _i64p), _p(sig, _u64p),
                                                  _p(sm, _f64p), _p(se, _i64p)))
    return delta, dist, sig, rc == SIGMA_OVERFLOW, sm, se


def exact_bc_w(g, w) -> np.ndarray:
    n, rp, col = _csr(g)
    wt = _wts(g, w)
    bc = np.empty(n, np.float64)
    _check(_load().orc_exact_bc_w(n, _p(rp, _i32p), _p(col, _i32p), _p(wt, _u32p), _p(bc, _f64p)))
    return bc


def uniform_sources_w(g, w, k: int, seed: int, qid: int) -> np.ndarray:
    n, rp, col = _csr(g)
    wt = _wts(g, w)
    est = np.empty(n, np.float64)
    _check(_load().orc_uniform_sources_w(n, _p(rp, _i32p), _p(col, _i32p), _p(wt, _u32p), k, seed, qid,
                                         _p(est, _f64p)))
    return est


def adaptive_sources_w(g, w, targets, c: float, cap: int, seed: int, qid: int):
    n, rp, col = _csr(g)
    wt = _wts(g, w)
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    T = tg.size
    est = np.empty(T, np.float64)
    k = np.empty(T, np.int64)
    S = np.empty(T, np.float64)
    st = np.empty(T, np.int32)
    tgp = tg if T else np.zeros(1, np.int32)
    _check(_load().orc_adaptive_sources_w(n, _p(rp, _i32p), _p(col, _i32p), _p(wt, _u32p), T, _p(tgp, _i32p),
                                          c, cap, seed, qid, _p(est, _f64p), _p(k, _i64p), _p(S, _f64p),
                                          _p(st, _i32p)))
    return dict(est=est, k=k, S=S, status=st)


# ------------------------------------------------ steps for parallel drivers --

class UniformAccumulator:
    """The exact per-vertex sums of the uniform estimate (``uniform_sources``),
    fed with dependency rows computed elsewhere (e.g. ``dependencies`` on many
    host cores at once). ``add_rows`` may be called for disjoint vertex ranges
    from several threads at the same time; ``estimate(k)`` rounds each sum once
    and returns (n*S)/k, exactly as ``uniform_sources`` does for the same rows."""

    def __init__(self, n: int):
        self.n = int(n)
        self._h = _load().orc_accs_new(self.n)
        if not self._h:
            raise MemoryError("oracle accumulators")

    def add_rows(self, rows, v0: int = 0, v1: int | None = None):
        rows = np.ascontiguousarray(rows, dtype=np.float64).reshape(-1, self.n)
        v1 = self.n if v1 is None else int(v1)
        _load().orc_accs_add_rows(self._h, self.n, int(v0), v1, _p(rows, _f64p), rows.shape[0])

    def estimate(self, k: int) -> np.ndarray:
        est = np.empty(self.n, np.float64)
        _load().orc_accs_uniform_est(self._h, self.n, int(k), _p(est, _f64p))
        return est

    def close(self):
        if self._h:
            _load().orc_accs_free(self._h)
            self._h = None

    def __del__(self):
        self.close()


def pair_sequence_multi(g, targets, seed: int, qid: int, i0: int, count: int) -> np.ndarray:
    """y[j, q]: the pair value of target j for draw i0+q (Algorithm 1), for all
    targets with one BFS from s per draw; row j equals ``pair_sequence`` for
    target j alone."""
    n, rp, col = _csr(g)
    t = np.ascontiguousarray(targets, dtype=np.int32)
    y = np.empty((t.shape[0], max(int(count), 0)), np.float64)
    _check(_load().orc_pair_sequence_multi(n, _p(rp, _i32p), _p(col, _i32p), t.shape[0], _p(t, _i32p),
                                           seed, qid, i0, count, _p(y, _f64p)))
    return y
