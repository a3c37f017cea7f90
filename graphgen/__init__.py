"""Seeded synthetic inputs shared by the CPU oracle, the CUDA library, the tests
and the benchmark.

This package holds input generation only -- graph families, the CSR normaliser
and target-set selection. None of the betweenness arithmetic lives here. The C
core is ``graphgen.c`` (integer-only counter-based hashing, so a given seed gives
the same graph on every host); :func:`build` compiles it with gcc.

Workload recipes (sizes, seeds) used by the benchmark and the tests live in
:mod:`graphgen.workloads`.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "_graphgen.so")
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile graphgen.c into _graphgen.so (in-tree) and return its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.gg_er_pairs.restype = ctypes.c_int64
        lib.gg_er_pairs.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                    _i32p, _i32p, ctypes.c_int64]
        lib.gg_er_m.restype = None
        lib.gg_er_m.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, _i32p, _i32p]
        lib.gg_rmat.restype = None
        lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, _i32p, _i32p]
        lib.gg_ba.restype = ctypes.c_int
        lib.gg_ba.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                              _i32p, _i32p]
        lib.gg_grid.restype = ctypes.c_int64
        lib.gg_grid.argtypes = [ctypes.c_int32, _i32p, _i32p]
        lib.gg_csr.restype = ctypes.c_int64
        lib.gg_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p, _i32p, _i32p,
                               ctypes.POINTER(_i32p)]
        lib.gg_free.restype = None
        lib.gg_free.argtypes = [ctypes.c_void_p]
        lib.gg_uniform_targets.restype = ctypes.c_int
        lib.gg_uniform_targets.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _i32p]
        lib.gg_degree_targets.restype = ctypes.c_int
        lib.gg_degree_targets.argtypes = [ctypes.c_int32, _i32p, ctypes.c_int32,
                                          ctypes.c_uint64, _i32p]
        lib.gg_edge_lengths.restype = None
        lib.gg_edge_lengths.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32)]
        lib.gg_rand.restype = ctypes.c_uint64
        lib.gg_rand.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_i32p)


class Graph:
    """Undirected unweighted graph in CSR form (int32 row_ptr[n+1], int32 col[nnz]).

    Rows are sorted ascending, with no self loops and no duplicates, and the
    adjacency is symmetric. ``nnz`` counts directed entries (2 per undirected edge).
    """

    def __init__(self, row_ptr: np.ndarray, col: np.ndarray, name: str = "graph"):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.name = name

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def neighbors(self, v: int) -> np.ndarray:
        return self.col[self.row_ptr[v]:self.row_ptr[v + 1]]

    def edges(self):
        """Undirected edge list (u < v) as an (m, 2) int array."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        keep = src < self.col
        return np.stack([src[keep], self.col[keep].astype(np.int64)], axis=1)

    def __repr__(self):
        return f"Graph({self.name}, n={self.n}, nnz={self.nnz})"


def from_edges(n: int, eu, ev, name: str = "graph") -> Graph:
    """Normalise an edge list (any orientation, loops/duplicates allowed) into CSR."""
    lib = _load()
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    assert eu.shape == ev.shape
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    colp = _i32p()
    nnz = lib.gg_csr(n, eu.shape[0], _p(eu), _p(ev), _p(row_ptr), ctypes.byref(colp))
    if nnz < 0:
        raise ValueError(f"gg_csr failed with code {nnz}")
    col = np.ctypeslib.as_array(colp, shape=(max(nnz, 1),))[:nnz].copy()
    lib.gg_free(ctypes.cast(colp, ctypes.c_void_p))
    return Graph(row_ptr, col, name)


def from_edges_directed(n: int, eu, ev, name: str = "digraph") -> Graph:
    """A directed CSR from an edge list u -> v: self loops and repeated edges
    dropped, each row (the out-neighbours) sorted; no symmetrisation."""
    eu = np.asarray(eu, dtype=np.int64)
    ev = np.asarray(ev, dtype=np.int64)
    keep = eu != ev
    key = np.unique(eu[keep] * n + ev[keep])
    src = (key // n).astype(np.int32)
    col = (key % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(row_ptr, src.astype(np.int64) + 1, 1)
    row_ptr = np.cumsum(row_ptr, dtype=np.int64).astype(np.int32)
    return Graph(row_ptr, col, name)


def directed_rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int) -> Graph:
    """R-MAT edges read as directed (row -> column quadrant), not symmetrised."""
    lib = _load()
    n = 1 << scale
    M = edge_factor * n
    eu = np.empty(M, np.int32)
    ev = np.empty(M, np.int32)
    lib.gg_rmat(scale, M, a, b, c, seed, _p(eu), _p(ev))
    return from_edges_directed(n, eu, ev, name=f"drmat_s{scale}_ef{edge_factor}_s{seed}")


def directed_er(n: int, avg_out_degree: float, seed: int) -> Graph:
    """Directed G(n, M): M = round(avg_out_degree * n) uniform ordered pairs."""
    lib = _load()
    M = int(round(avg_out_degree * n))
    eu = np.empty(M, np.int32)
    ev = np.empty(M, np.int32)
    lib.gg_er_m(n, M, seed, _p(eu), _p(ev))
    return from_edges_directed(n, eu, ev, name=f"der_n{n}_d{avg_out_degree:g}_s{seed}")


def directed_grid(side: int) -> Graph:
    """side x side lattice with edges pointing right and down only (from the
    corner 0, sigma to (i, j) is the binomial C(i+j, i))."""
    v = np.arange(side * side, dtype=np.int64)
    i, j = v // side, v % side
    right = v[j + 1 < side]
    down = v[i + 1 < side]
    eu = np.concatenate([right, down])
    ev = np.concatenate([right + 1, down + side])
    return from_edges_directed(side * side, eu, ev, name=f"dgrid_{side}")


def erdos_renyi(n: int, avg_degree: float, seed: int, pairwise=None) -> Graph:
    """G(n, p) with p = avg_degree/(n-1).

    With pairwise (default: n <= 32768) every pair i<j is an exact Bernoulli(p)
    trial. Otherwise the G(n, M) form is used: M = round(p*n(n-1)/2) uniform
    endpoint pairs, then self loops and repeats are dropped.
    """
    lib = _load()
    p = avg_degree / (n - 1)
    if pairwise is None:
        pairwise = n <= 32768
    if pairwise:
        cap = int(p * n * (n - 1) / 2 * 1.5) + 1024
        eu = np.empty(cap, np.int32)
        ev = np.empty(cap, np.int32)
        m = lib.gg_er_pairs(n, p, seed, _p(eu), _p(ev), cap)
        if m > cap:
            eu = np.empty(m, np.int32)
            ev = np.empty(m, np.int32)
            m = lib.gg_er_pairs(n, p, seed, _p(eu), _p(ev), m)
        eu, ev = eu[:m], ev[:m]
    else:
        M = int(round(p * n * (n - 1) / 2))
        eu = np.empty(M, np.int32)
        ev = np.empty(M, np.int32)
        lib.gg_er_m(n, M, seed, _p(eu), _p(ev))
    return from_edges(n, eu, ev, name=f"er_n{n}_d{avg_degree:g}_s{seed}")


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int) -> Graph:
    """R-MAT with 2^scale vertices and edge_factor*2^scale generated edges."""
    lib = _load()
    n = 1 << scale
    M = edge_factor * n
    eu = np.empty(M, np.int32)
    ev = np.empty(M, np.int32)
    lib.gg_rmat(scale, M, a, b, c, seed, _p(eu), _p(ev))
    return from_edges(n, eu, ev, name=f"rmat_s{scale}_ef{edge_factor}_s{seed}")


def barabasi_albert(n: int, m: int, seed: int, m0: int = 5) -> Graph:
    lib = _load()
    M = m0 * (m0 - 1) // 2 + (n - m0) * m
    eu = np.empty(M, np.int32)
    ev = np.empty(M, np.int32)
    rc = lib.gg_ba(n, m0, m, seed, _p(eu), _p(ev))
    if rc != 0:
        raise ValueError(f"gg_ba failed with code {rc}")
    return from_edges(n, eu, ev, name=f"ba_n{n}_m{m}_s{seed}")


def grid(side: int) -> Graph:
    lib = _load()
    M = max(2 * side * (side - 1), 1)
    eu = np.empty(M, np.int32)
    ev = np.empty(M, np.int32)
    m = lib.gg_grid(side, _p(eu), _p(ev))
    return from_edges(side * side, eu[:m], ev[:m], name=f"grid_{side}")


def uneven_set(count: int = 256, base_seed: int = 6, n_lo: int = 2000, n_hi: int = 200000):
    """The uneven multi-graph workload: `count` graphs with sizes log-uniform in
    [n_lo, n_hi], each an Erdos-Renyi graph (G(n, M) form, average degree
    uniform in 4..16), an R-MAT graph (2^round(log2 n) vertices, edge factor 8,
    a=0.57 b=0.19 c=0.19) or a 2D grid of side floor(sqrt(n)), the family and
    every parameter drawn from the generator's hash of (base_seed, stream, i).
    Returns a list of (family, Graph)."""
    out = []
    lo, hi = math.log(n_lo), math.log(n_hi)
    for i in range(count):
        u = (rand64(base_seed, 1, i) >> 11) / float(1 << 53)
        n = int(round(math.exp(lo + u * (hi - lo))))
        fam = rand64(base_seed, 2, i) % 3
        seed = rand64(base_seed, 3, i) & 0x7FFFFFFF
        if fam == 0:
            deg = 4 + rand64(base_seed, 4, i) % 13
            out.append(("er", erdos_renyi(n, float(deg), seed, pairwise=False)))
        elif fam == 1:
            out.append(("rmat", rmat(max(1, int(round(math.log2(n)))), 8, 0.57, 0.19, 0.19, seed)))
        else:
            out.append(("grid", grid(max(1, int(math.isqrt(n))))))
    return out


def uniform_targets(n: int, T: int, seed: int) -> np.ndarray:
    """T distinct vertices, uniform over [0, n)."""
    lib = _load()
    out = np.empty(T, np.int32)
    if lib.gg_uniform_targets(n, T, seed, _p(out)) != 0:
        raise ValueError("invalid target request")
    return out


def degree_targets(g: Graph, T: int, seed: int) -> np.ndarray:
    """T distinct vertices drawn with probability proportional to degree."""
    lib = _load()
    out = np.empty(T, np.int32)
    if lib.gg_degree_targets(g.n, _p(g.row_ptr), T, seed, _p(out)) != 0:
        raise ValueError("invalid target request")
    return out


def rand64(seed: int, stream: int, idx: int) -> int:
    """The generator's 64-bit hash (exposed for tests and derived seeds)."""
    return int(_load().gg_rand(seed, stream, idx))


def edge_lengths(g: Graph, lo: int, hi: int, seed: int, symmetric: bool = True) -> np.ndarray:
    """uint32 lengths in [lo, hi], one per CSR entry, from a hash of the edge
    (the unordered pair when symmetric, so both rows of an undirected edge
    agree) and the seed."""
    if not (1 <= lo <= hi < 2**32):
        raise ValueError("need 1 <= lo <= hi < 2^32")
    lib = _load()
    w = np.empty(max(1, g.col.shape[0]), np.uint32)
    lib.gg_edge_lengths(g.n, _p(g.row_ptr), _p(g.col) if g.col.size else _p(np.zeros(1, np.int32)), lo, hi,
                        seed, 1 if symmetric else 0, w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return w[: g.col.shape[0]]
