"""ctypes binding of include/bc.h: argument marshalling and status checks only.

Every function named ``bc_*`` here wraps the C entry point of the same name.
Arrays are numpy; outputs are allocated here and returned. A negative status
raises :class:`BCError` carrying the code and ``bc_last_error``'s message.
"""
from __future__ import annotations

import ctypes
import os
from types import SimpleNamespace

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libbcgb300.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_1608_04472_gb300.build` "
        "(nvcc, sm_103a). There is no CPU fallback.")
_lib = ctypes.CDLL(LIB_PATH)

BC_OK = 0
BC_STOPPED = 0
BC_CAPPED = 1
BC_UNDIRECTED = 1
BC_VALIDATE = 2
BC_DIRECTED = 4
BC_NORMALIZE = 8
BC_PENDING = 1
BC_QUERY_SOURCES = 1
BC_QUERY_PAIRS = 2
BC_QUERY_UNIFORM = 3
STATUS_NAMES = {
    -1: "BC_E_INVALID", -2: "BC_E_NOMEM", -3: "BC_E_TOO_LARGE", -4: "BC_E_BAD_GRAPH",
    -5: "BC_E_DEVICE", -6: "BC_E_DEVICE_TIMEOUT", -7: "BC_E_CANCELLED",
    -8: "BC_E_UNKNOWN_HANDLE", -9: "BC_E_SIGMA_OVERFLOW", -10: "BC_E_RANGE",
}

_vp = ctypes.c_void_p
_i32, _i64, _u32, _u64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
_i32p = ctypes.POINTER(_i32)
_i64p = ctypes.POINTER(_i64)
_u64p = ctypes.POINTER(_u64)
_f64p = ctypes.POINTER(_f64)


class bc_options(ctypes.Structure):
    _fields_ = [("batch_width", _i32), ("reserved0", _i32), ("stream", _vp)]


class bc_query_stats(ctypes.Structure):
    _fields_ = [("queue_ms", _f64), ("run_ms", _f64), ("samples", _i64), ("batches", _i64)]


class bc_query(ctypes.Structure):
    _fields_ = [("kind", _i32), ("T", _i32), ("graph", _i64), ("targets", _i32p), ("c", _f64),
                ("cap", _i64), ("k", _i64), ("seed", _u64), ("qid", _u64), ("threshold_scale", _f64),
                ("est", _f64p), ("k_out", _i64p), ("S_out", _f64p), ("stop_status", _i32p),
                ("stats", ctypes.POINTER(bc_query_stats))]


class bc_tuning(ctypes.Structure):
    _fields_ = [("batch_width", _i32), ("heavy_degree", _i32), ("segment", _i32), ("packed_max_lanes", _i32),
                ("packed_min_preds", _i32), ("bwd_variant", _i32), ("heavy_lane", _i32), ("push_div", _i32),
                ("deep_levels", _i32), ("reserved0", _i32), ("trial_ms", _f64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved0"}


TUNING_FIELDS = tuple(name for name, _ in bc_tuning._fields_ if name not in ("reserved0", "trial_ms"))


class bc_stats(ctypes.Structure):
    _fields_ = [("launches", _i64), ("samples", _i64), ("batches", _i64), ("dag_edges", _i64),
                ("reached", _i64),
                ("n_kernels", _i32), ("pair_fallbacks", _i32), ("kernel_name", (ctypes.c_char * 32) * 16),
                ("kernel_launches", _i64 * 16), ("kernel_ms", _f64 * 16)]


_SIGS = {
    "bc_create": (_i32, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(bc_options)]),
    "bc_destroy": (None, [_vp]),
    "bc_last_error": (ctypes.c_char_p, [_vp]),
    "bc_set_batch_width": (_i32, [_vp, _i32]),
    "bc_graph_load_csr": (_i32, [_vp, _i32, _i32p, _i32p, _i64, _u32, _i64p]),
    "bc_graph_load_csr_weighted": (_i32, [_vp, _i32, _i32p, _i32p, ctypes.POINTER(_u32), _i64, _u32, _i64p]),
    "bc_graph_free": (_i32, [_vp, _i64]),
    "bc_graph_info": (_i32, [_vp, _i64, _i32p, _i64p]),
    "bc_source_dependencies": (_i32, [_vp, _i64, _i32p, _i32, _f64p, _i32p, _u64p]),
    "bc_source_dependencies_ext": (_i32, [_vp, _i64, _i32p, _i32, _f64p, _i32p, _f64p, _i32p, _i32p]),
    "bc_source_dependencies_weighted": (_i32, [_vp, _i64, _i32p, _i32, _f64p, _i64p, _u64p, _f64p, _i32p, _i32p]),
    "bc_uniform_sources_multi": (_i32, [_vp, _i32, _i64p, _i64p, _u64p, _u64p, _f64p]),
    "bc_exact": (_i32, [_vp, _i64, _f64p]),
    "bc_uniform_sources": (_i32, [_vp, _i64, _i64, _u64, _u64, _f64p]),
    "bc_adaptive_sources": (_i32, [_vp, _i64, _i32p, _i32, _f64, _i64, _u64, _u64, _f64p, _i64p,
                                   _f64p, _i32p]),
    "bc_adaptive_pairs": (_i32, [_vp, _i64, _i32p, _i32, _f64, _i64, _u64, _u64, _f64, _f64p, _i64p,
                                 _f64p, _i32p]),
    "bc_submit": (_i32, [_vp, ctypes.POINTER(bc_query), _i64p]),
    "bc_poll": (_i32, [_vp, _i64, _i64]),
    "bc_cancel": (_i32, [_vp, _i64]),
    "bc_server_limits": (_i32, [_vp, _i32, _i64]),
    "bc_source_dependencies_noalloc": (_i32, [ctypes.c_int, _vp, _vp, _i32, _i64, _vp, _i32, _vp, _vp]),
    "bc_draw_sources": (_i32, [_vp, _u64, _u64, _u64, _i64, _i32, _i32p]),
    "bc_draw_pairs": (_i32, [_vp, _u64, _u64, _u64, _i64, _i32, _i32p, _i32p]),
    "bc_exact_sum": (_i32, [_vp, _f64p, _i64, _f64p]),
    "bc_target_dependencies": (_i32, [_vp, _i64, _i32p, _i32, _u64, _u64, _i64, _i64, _f64p]),
    "bc_pair_values": (_i32, [_vp, _i64, _i32p, _i32, _u64, _u64, _i64, _i64, _f64p]),
    "bc_uniform_partial": (_i32, [_vp, _i64, _u64, _u64, _i64, _i64, _i64p]),
    "bc_acc_add_rows": (_i32, [_i32, _f64p, _i64, _i64p]),
    "bc_acc_estimate": (_i32, [_i32, _i64p, _i64, _f64p]),
    "bc_scan_block": (_i32, [_i32, _f64p, _i32, _i64, _f64, _f64, _f64, _f64p, _i64p, _i32p, _f64p, _i32p, _i32p]),
    "bc_autotune": (_i32, [_vp, _i64, _i64, _u64, ctypes.POINTER(bc_tuning)]),
    "bc_get_tuning": (_i32, [_vp, _i64, ctypes.POINTER(bc_tuning)]),
    "bc_set_tuning": (_i32, [_vp, _i64, ctypes.POINTER(bc_tuning)]),
    "bc_set_profiling": (_i32, [_vp, _i32]),
    "bc_get_stats": (_i32, [_vp, ctypes.POINTER(bc_stats)]),
    "bc_reset_stats": (_i32, [_vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class BCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ck(ctx, rc):
    if rc < 0:
        msg = _lib.bc_last_error(ctx)
        raise BCError(rc, msg.decode() if msg else "")
    return rc


def _p(a, t):
    return a.ctypes.data_as(t)


def _i32arr(x):
    return np.ascontiguousarray(x, dtype=np.int32)


# ------------------------------------------------------- same-name functions --

def bc_create(device: int = 0, batch_width: int = 0, stream: int | None = None):
    opt = bc_options(batch_width, 0, stream or None)
    out = _vp()
    rc = _lib.bc_create(ctypes.byref(out), device, ctypes.byref(opt))
    if rc < 0:
        raise BCError(rc, "bc_create failed (no CUDA device or bad option)")
    return out


def bc_destroy(ctx):
    _lib.bc_destroy(ctx)


def bc_last_error(ctx) -> str:
    return _lib.bc_last_error(ctx).decode()


def bc_set_batch_width(ctx, width: int):
    _ck(ctx, _lib.bc_set_batch_width(ctx, width))


def bc_graph_load_csr(ctx, row_ptr, col, flags: int = BC_UNDIRECTED) -> int:
    rp = _i32arr(row_ptr)
    cl = _i32arr(col)
    n = rp.shape[0] - 1
    cl_ = cl if cl.size else np.zeros(1, np.int32)
    h = _i64()
    _ck(ctx, _lib.bc_graph_load_csr(ctx, n, _p(rp, _i32p), _p(cl_, _i32p), int(cl.size), flags,
                                    ctypes.byref(h)))
    return int(h.value)


def bc_graph_load_csr_weighted(ctx, row_ptr, col, lengths, flags: int = BC_UNDIRECTED) -> int:
    rp = _i32arr(row_ptr)
    cl = _i32arr(col)
    wl = np.ascontiguousarray(lengths, dtype=np.uint32)
    if wl.shape[0] != cl.shape[0]:
        raise ValueError("one length per CSR entry")
    n = rp.shape[0] - 1
    cl_ = cl if cl.size else np.zeros(1, np.int32)
    wl_ = wl if wl.size else np.ones(1, np.uint32)
    h = _i64()
    _ck(ctx, _lib.bc_graph_load_csr_weighted(ctx, n, _p(rp, _i32p), _p(cl_, _i32p),
                                             wl_.ctypes.data_as(ctypes.POINTER(_u32)), int(cl.size), flags,
                                             ctypes.byref(h)))
    return int(h.value)


def bc_graph_free(ctx, g: int):
    _ck(ctx, _lib.bc_graph_free(ctx, g))


def bc_graph_info(ctx, g: int):
    n, nnz = _i32(), _i64()
    _ck(ctx, _lib.bc_graph_info(ctx, g, ctypes.byref(n), ctypes.byref(nnz)))
    return int(n.value), int(nnz.value)


def bc_source_dependencies(ctx, g: int, sources, want_dist: bool = False, want_sigma: bool = False):
    n, _ = bc_graph_info(ctx, g)
    src = _i32arr(sources)
    cnt = src.size
    delta = np.zeros((cnt, n), np.float64)
    dist = np.zeros((cnt, n), np.int32) if want_dist else None
    sigma = np.zeros((cnt, n), np.uint64) if want_sigma else None
    srcp = src if cnt else np.zeros(1, np.int32)
    _ck(ctx, _lib.bc_source_dependencies(
        ctx, g, _p(srcp, _i32p), cnt, _p(delta, _f64p) if cnt else None,
        _p(dist, _i32p) if dist is not None and cnt else None,
        _p(sigma, _u64p) if sigma is not None and cnt else None))
    return delta, dist, sigma


def bc_source_dependencies_ext(ctx, g: int, sources):
    """(delta [count][n], dist [count][n], sigma mantissa [count][n], sigma exponent
    [count][n], tier [count]); sigma = mantissa * 2**exponent, tier 1 = the
    source was computed in the extended form."""
    n, _ = bc_graph_info(ctx, g)
    src = _i32arr(sources)
    cnt = src.size
    delta = np.zeros((cnt, n), np.float64)
    dist = np.zeros((cnt, n), np.int32)
    sm = np.zeros((cnt, n), np.float64)
    se = np.zeros((cnt, n), np.int32)
    tier = np.zeros(cnt, np.int32)
    if cnt:
        _ck(ctx, _lib.bc_source_dependencies_ext(ctx, g, _p(src, _i32p), cnt, _p(delta, _f64p), _p(dist, _i32p),
                                                 _p(sm, _f64p), _p(se, _i32p), _p(tier, _i32p)))
    return delta, dist, sm, se, tier


def bc_source_dependencies_weighted(ctx, g: int, sources):
    """(delta [count][n], dist int64 [count][n], sigma [count][n], sigma mantissa,
    sigma exponent, tier [count]) from the weighted engine (unit lengths on a
    graph without lengths)."""
    n, _ = bc_graph_info(ctx, g)
    src = _i32arr(sources)
    cnt = src.size
    delta = np.zeros((cnt, n), np.float64)
    dist = np.zeros((cnt, n), np.int64)
    sig = np.zeros((cnt, n), np.uint64)
    sm = np.zeros((cnt, n), np.float64)
    se = np.zeros((cnt, n), np.int32)
    tier = np.zeros(cnt, np.int32)
    if cnt:
        _ck(ctx, _lib.bc_source_dependencies_weighted(ctx, g, _p(src, _i32p), cnt, _p(delta, _f64p),
                                                      _p(dist, _i64p), _p(sig, _u64p), _p(sm, _f64p),
                                                      _p(se, _i32p), _p(tier, _i32p)))
    return delta, dist, sig, sm, se, tier


def bc_uniform_sources_multi(ctx, graphs, k, seeds, qids):
    """Uniform estimates for several graphs in one persistent launch; returns a
    list of per-graph arrays (graph i: n_i values)."""
    hs = np.ascontiguousarray(graphs, dtype=np.int64)
    G = hs.size
    kk = np.ascontiguousarray(np.broadcast_to(np.asarray(k, dtype=np.int64), (G,)))
    ss = np.ascontiguousarray(np.broadcast_to(np.asarray(seeds, dtype=np.uint64), (G,)))
    qq = np.ascontiguousarray(np.broadcast_to(np.asarray(qids, dtype=np.uint64), (G,)))
    ns = [bc_graph_info(ctx, int(h))[0] for h in hs.tolist()]
    out = np.empty(max(1, sum(ns)), np.float64)
    _ck(ctx, _lib.bc_uniform_sources_multi(ctx, G, _p(hs, _i64p), _p(kk, _i64p), _p(ss, _u64p), _p(qq, _u64p),
                                           _p(out, _f64p)))
    res, off = [], 0
    for n in ns:
        res.append(out[off:off + n].copy())
        off += n
    return res


def bc_exact(ctx, g: int) -> np.ndarray:
    n, _ = bc_graph_info(ctx, g)
    out = np.empty(n, np.float64)
    _ck(ctx, _lib.bc_exact(ctx, g, _p(out, _f64p)))
    return out


def bc_uniform_sources(ctx, g: int, k: int, seed: int, qid: int) -> np.ndarray:
    n, _ = bc_graph_info(ctx, g)
    out = np.empty(n, np.float64)
    _ck(ctx, _lib.bc_uniform_sources(ctx, g, k, seed, qid, _p(out, _f64p)))
    return out


def _target_outputs(T):
    return (np.zeros(max(T, 1), np.float64), np.zeros(max(T, 1), np.int64),
            np.zeros(max(T, 1), np.float64), np.zeros(max(T, 1), np.int32))


def bc_adaptive_sources(ctx, g: int, targets, c: float, cap: int, seed: int, qid: int):
    tg = _i32arr(targets)
    T = tg.size
    est, k, S, st = _target_outputs(T)
    tgp = tg if T else np.zeros(1, np.int32)
    _ck(ctx, _lib.bc_adaptive_sources(ctx, g, _p(tgp, _i32p), T, c, cap, seed, qid, _p(est, _f64p),
                                      _p(k, _i64p), _p(S, _f64p), _p(st, _i32p)))
    return dict(est=est[:T], k=k[:T], S=S[:T], status=st[:T])


def bc_adaptive_pairs(ctx, g: int, targets, c: float, cap: int, seed: int, qid: int,
                      threshold_scale: float = 1.0):
    tg = _i32arr(targets)
    T = tg.size
    est, k, S, st = _target_outputs(T)
    tgp = tg if T else np.zeros(1, np.int32)
    _ck(ctx, _lib.bc_adaptive_pairs(ctx, g, _p(tgp, _i32p), T, c, cap, seed, qid, threshold_scale,
                                    _p(est, _f64p), _p(k, _i64p), _p(S, _f64p), _p(st, _i32p)))
    return dict(est=est[:T], k=k[:T], S=S[:T], status=st[:T])


class Ticket:
    """A submitted query: owns its input copy and output buffers until polled."""

    def __init__(self, kind, T, n):
        self.kind = kind
        m = n if kind == BC_QUERY_UNIFORM else max(T, 1)
        self.est = np.zeros(m, np.float64)
        self.k = np.zeros(max(T, 1), np.int64)
        self.S = np.zeros(max(T, 1), np.float64)
        self.status = np.zeros(max(T, 1), np.int32)
        self.stats = bc_query_stats()
        self.T = T
        self.id = None
        self.targets = None
        self.result = None

    def outputs(self):
        if self.kind == BC_QUERY_UNIFORM:
            return dict(est=self.est)
        T = self.T
        return dict(est=self.est[:T], k=self.k[:T], S=self.S[:T], status=self.status[:T])

    def stats_dict(self):
        s = self.stats
        return dict(queue_ms=s.queue_ms, run_ms=s.run_ms, samples=int(s.samples), batches=int(s.batches))


def bc_submit(ctx, g: int, kind: int, targets=None, c: float = 1.0, cap: int = 1, k: int = 0,
              seed: int = 0, qid: int = 0, threshold_scale: float = 1.0) -> Ticket:
    n, _ = bc_graph_info(ctx, g)
    tg = _i32arr(targets if targets is not None else [])
    T = int(tg.size)
    tk = Ticket(kind, T, n)
    tk.targets = tg if T else np.zeros(1, np.int32)
    q = bc_query(kind, T, g, _p(tk.targets, _i32p), c, cap, k, seed, qid, threshold_scale,
                 _p(tk.est, _f64p), _p(tk.k, _i64p), _p(tk.S, _f64p), _p(tk.status, _i32p),
                 ctypes.pointer(tk.stats))
    t = _i64()
    _ck(ctx, _lib.bc_submit(ctx, ctypes.byref(q), ctypes.byref(t)))
    tk.id = int(t.value)
    return tk


def bc_poll(ctx, ticket: Ticket, timeout_us: int = -1) -> int:
    """Returns BC_OK (outputs ready) or BC_PENDING; raises BCError on a failed query."""
    rc = _lib.bc_poll(ctx, ticket.id, timeout_us)
    if rc == BC_PENDING:
        return rc
    ticket.result = rc
    _ck(ctx, rc)
    return rc


def bc_cancel(ctx, ticket: Ticket):
    _ck(ctx, _lib.bc_cancel(ctx, ticket.id))


def bc_server_limits(ctx, max_active: int = 0, mem_budget_bytes: int = 0):
    _ck(ctx, _lib.bc_server_limits(ctx, max_active, mem_budget_bytes))


BC_NOALLOC_MAX_VERTICES = 262144


def bc_source_dependencies_noalloc(device: int, d_row_ptr: int, d_col: int, n: int, nnz: int,
                                   d_sources: int, count: int, d_delta_out: int, stream: int = 0) -> int:
    """Allocation-free per-source dependencies on caller-owned DEVICE buffers
    (addresses as ints, e.g. torch tensors' data_ptr()). Returns the status code;
    there is no context, so there is no error message."""
    return int(_lib.bc_source_dependencies_noalloc(device, d_row_ptr or None, d_col or None, n, nnz,
                                                   d_sources or None, count, d_delta_out or None,
                                                   stream or None))


def bc_draw_sources(ctx, seed: int, qid: int, i0: int, count: int, n: int) -> np.ndarray:
    out = np.zeros(max(count, 1), np.int32)
    _ck(ctx, _lib.bc_draw_sources(ctx, seed, qid, i0, count, n, _p(out, _i32p)))
    return out[:count]


def bc_draw_pairs(ctx, seed: int, qid: int, i0: int, count: int, n: int):
    s = np.zeros(max(count, 1), np.int32)
    t = np.zeros(max(count, 1), np.int32)
    _ck(ctx, _lib.bc_draw_pairs(ctx, seed, qid, i0, count, n, _p(s, _i32p), _p(t, _i32p)))
    return s[:count], t[:count]


def bc_exact_sum(ctx, x) -> float:
    a = np.ascontiguousarray(x, dtype=np.float64)
    out = _f64()
    ap = a if a.size else np.zeros(1, np.float64)
    _ck(ctx, _lib.bc_exact_sum(ctx, _p(ap, _f64p), a.size, ctypes.byref(out)))
    return float(out.value)


def bc_target_dependencies(ctx, g: int, targets, seed: int, qid: int, i0: int, count: int) -> np.ndarray:
    """[T][count] block of delta_{s_i}(v_j) for draws i0 .. i0+count-1."""
    t = _i32arr(targets)
    out = np.zeros((t.size, max(int(count), 0)), np.float64)
    tp = t if t.size else np.zeros(1, np.int32)
    op = out if out.size else np.zeros(1, np.float64)
    _ck(ctx, _lib.bc_target_dependencies(ctx, g, _p(tp, _i32p), t.size, seed, qid, i0, int(count), _p(op, _f64p)))
    return out


def bc_pair_values(ctx, g: int, targets, seed: int, qid: int, i0: int, count: int) -> np.ndarray:
    """[T][count] block of Algorithm 1's per-draw pair values for draws i0 .. i0+count-1."""
    t = _i32arr(targets)
    out = np.zeros((t.size, max(int(count), 0)), np.float64)
    tp = t if t.size else np.zeros(1, np.int32)
    op = out if out.size else np.zeros(1, np.float64)
    _ck(ctx, _lib.bc_pair_values(ctx, g, _p(tp, _i32p), t.size, seed, qid, i0, int(count), _p(op, _f64p)))
    return out


def bc_uniform_partial(ctx, g: int, seed: int, qid: int, i0: int, count: int, parts: np.ndarray) -> np.ndarray:
    """Adds the exact sums of draws i0 .. i0+count-1 into parts (int64 [n][6], in place)."""
    if parts.dtype != np.int64 or not parts.flags.c_contiguous:
        raise ValueError("parts must be a C-contiguous int64 array [n][6]")
    _ck(ctx, _lib.bc_uniform_partial(ctx, g, seed, qid, i0, int(count), _p(parts, _i64p)))
    return parts


def _ck_host(rc, what):
    if rc < 0:
        raise BCError(rc, what)
    return rc


def bc_acc_add_rows(rows, parts: np.ndarray) -> np.ndarray:
    """Adds rows (count x n doubles) exactly into parts (int64 [n][6], in place)."""
    if parts.dtype != np.int64 or not parts.flags.c_contiguous:
        raise ValueError("parts must be a C-contiguous int64 array [n][6]")
    n = parts.shape[0]
    r = np.ascontiguousarray(rows, dtype=np.float64).reshape(-1, n)
    rp = r if r.size else np.zeros(1, np.float64)
    _ck_host(_lib.bc_acc_add_rows(n, _p(rp, _f64p), r.shape[0], _p(parts, _i64p)), "bc_acc_add_rows")
    return parts


def bc_acc_estimate(parts: np.ndarray, k: int) -> np.ndarray:
    parts = np.ascontiguousarray(parts, dtype=np.int64)
    n = parts.shape[0]
    est = np.empty(n, np.float64)
    _ck_host(_lib.bc_acc_estimate(n, _p(parts, _i64p), int(k), _p(est, _f64p)), "bc_acc_estimate")
    return est


def bc_scan_block(block, i0: int, cn: float, threshold_scale: float, n_scale: float, state) -> int:
    """Stop scan of one [T][W] block in draw order; state (S, k, done, est,
    status: numpy arrays of T) is updated in place; returns targets not done."""
    b = np.ascontiguousarray(block, dtype=np.float64)
    S, k, done, est, status = state
    T = S.shape[0]
    W = b.shape[1] if b.ndim == 2 else 0
    bp = b if b.size else np.zeros(1, np.float64)
    rem = _i32()
    _ck_host(_lib.bc_scan_block(T, _p(bp, _f64p), W, int(i0), float(cn), float(threshold_scale), float(n_scale),
                                _p(S, _f64p), _p(k, _i64p), _p(done, _i32p), _p(est, _f64p), _p(status, _i32p),
                                ctypes.byref(rem)), "bc_scan_block")
    return int(rem.value)


def bc_autotune(ctx, g: int, k: int = 256, seed: int = 1) -> dict:
    t = bc_tuning()
    _ck(ctx, _lib.bc_autotune(ctx, g, int(k), seed, ctypes.byref(t)))
    return t.as_dict()


def bc_get_tuning(ctx, g: int) -> dict:
    t = bc_tuning()
    _ck(ctx, _lib.bc_get_tuning(ctx, g, ctypes.byref(t)))
    return t.as_dict()


def bc_set_tuning(ctx, g: int, tuning: dict):
    t = bc_tuning()
    for name in TUNING_FIELDS:
        setattr(t, name, int(tuning[name]))
    _ck(ctx, _lib.bc_set_tuning(ctx, g, ctypes.byref(t)))


def bc_set_profiling(ctx, on: bool):
    _ck(ctx, _lib.bc_set_profiling(ctx, 1 if on else 0))


def bc_get_stats(ctx) -> dict:
    s = bc_stats()
    _ck(ctx, _lib.bc_get_stats(ctx, ctypes.byref(s)))
    kern = {}
    for i in range(s.n_kernels):
        name = bytes(s.kernel_name[i]).split(b"\0", 1)[0].decode()
        kern[name] = dict(launches=int(s.kernel_launches[i]), ms=float(s.kernel_ms[i]))
    return dict(launches=int(s.launches), samples=int(s.samples), batches=int(s.batches),
                dag_edges=int(s.dag_edges), reached=int(s.reached), pair_fallbacks=int(s.pair_fallbacks),
                kernels=kern)


def bc_reset_stats(ctx):
    _ck(ctx, _lib.bc_reset_stats(ctx))


capi = SimpleNamespace(**{name: globals()[name] for name in _SIGS})


# ------------------------------------------------------------ object wrapper --

class Context:
    """Owns one bc_ctx (one CUDA device) and the graphs loaded into it."""

    def __init__(self, device: int = 0, batch_width: int = 0, stream: int | None = None):
        self.ptr = bc_create(device, batch_width, stream)
        self.graphs: set[int] = set()

    def close(self):
        if self.ptr:
            bc_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_graph(self, row_ptr, col, validate: bool = False, directed: bool = False, lengths=None,
                   normalize: bool = False) -> int:
        flags = ((BC_DIRECTED if directed else BC_UNDIRECTED) | (BC_VALIDATE if validate else 0)
                 | (BC_NORMALIZE if normalize else 0))
        if lengths is None:
            h = bc_graph_load_csr(self.ptr, row_ptr, col, flags)
        else:
            h = bc_graph_load_csr_weighted(self.ptr, row_ptr, col, lengths, flags)
        self.graphs.add(h)
        return h

    def free_graph(self, g: int):
        bc_graph_free(self.ptr, g)
        self.graphs.discard(g)

    def set_batch_width(self, w: int):
        bc_set_batch_width(self.ptr, w)

    def source_dependencies(self, g, sources, want_dist=False, want_sigma=False):
        return bc_source_dependencies(self.ptr, g, sources, want_dist, want_sigma)

    def source_dependencies_ext(self, g, sources):
        return bc_source_dependencies_ext(self.ptr, g, sources)

    def source_dependencies_weighted(self, g, sources):
        return bc_source_dependencies_weighted(self.ptr, g, sources)

    def uniform_sources_multi(self, graphs, k, seeds, qids):
        return bc_uniform_sources_multi(self.ptr, graphs, k, seeds, qids)

    def exact(self, g):
        return bc_exact(self.ptr, g)

    def uniform_sources(self, g, k, seed, qid):
        return bc_uniform_sources(self.ptr, g, k, seed, qid)

    def adaptive_sources(self, g, targets, c, cap, seed, qid):
        return bc_adaptive_sources(self.ptr, g, targets, c, cap, seed, qid)

    def adaptive_pairs(self, g, targets, c, cap, seed, qid, threshold_scale=1.0):
        return bc_adaptive_pairs(self.ptr, g, targets, c, cap, seed, qid, threshold_scale)

    def draw_sources(self, seed, qid, i0, count, n):
        return bc_draw_sources(self.ptr, seed, qid, i0, count, n)

    def draw_pairs(self, seed, qid, i0, count, n):
        return bc_draw_pairs(self.ptr, seed, qid, i0, count, n)

    def exact_sum(self, x):
        return bc_exact_sum(self.ptr, x)

    def submit(self, g, kind, targets=None, c=1.0, cap=1, k=0, seed=0, qid=0, threshold_scale=1.0):
        return bc_submit(self.ptr, g, kind, targets, c, cap, k, seed, qid, threshold_scale)

    def poll(self, ticket, timeout_us=-1):
        return bc_poll(self.ptr, ticket, timeout_us)

    def cancel(self, ticket):
        bc_cancel(self.ptr, ticket)

    def server_limits(self, max_active=0, mem_budget_bytes=0):
        bc_server_limits(self.ptr, max_active, mem_budget_bytes)

    def target_dependencies(self, g, targets, seed, qid, i0, count):
        return bc_target_dependencies(self.ptr, g, targets, seed, qid, i0, count)

    def pair_values(self, g, targets, seed, qid, i0, count):
        return bc_pair_values(self.ptr, g, targets, seed, qid, i0, count)

    def uniform_partial(self, g, seed, qid, i0, count, parts):
        return bc_uniform_partial(self.ptr, g, seed, qid, i0, count, parts)

    def autotune(self, g, k=256, seed=1):
        return bc_autotune(self.ptr, g, k, seed)

    def get_tuning(self, g):
        return bc_get_tuning(self.ptr, g)

    def set_tuning(self, g, tuning):
        bc_set_tuning(self.ptr, g, tuning)

    def set_profiling(self, on: bool):
        bc_set_profiling(self.ptr, on)

    def stats(self):
        return bc_get_stats(self.ptr)

    def reset_stats(self):
        bc_reset_stats(self.ptr)
