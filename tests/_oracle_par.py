"""Runs the CPU oracle on every host core, for parity checks at full size.

The oracle is single-threaded C called through ctypes, which releases the
interpreter lock, so a thread pool runs one oracle call per core. Nothing here
does arithmetic of the method itself: rows come from ``oracle.dependencies`` and
``oracle.pair_sequence_multi``, exact sums from ``oracle.UniformAccumulator``;
the stop-rule replays restate Sec. 4 steps 2-3 and Algorithm 1's loop in plain
Python doubles (one rounding per operation, as the oracle's C does), the same
replays the CPU pins check against ``oracle.adaptive_sources`` and
``oracle.adaptive_pairs``.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


def workers() -> int:
    return max(1, os.cpu_count() or 1)


def dependency_rows(g, sources, pool) -> np.ndarray:
    """Oracle delta rows [len(sources)][n], one oracle call per source."""
    rows = list(pool.map(lambda s: oracle.dependencies(g, int(s))[0], sources))
    return np.stack(rows) if rows else np.zeros((0, g.n))


def add_rows_parallel(acc, rows, pool, parts: int):
    """Adds rows into the accumulator, vertex range by vertex range in parallel."""
    n = acc.n
    cuts = np.linspace(0, n, parts + 1).astype(np.int64)
    list(pool.map(lambda i: acc.add_rows(rows, int(cuts[i]), int(cuts[i + 1])), range(parts)))


def uniform_estimate(g, sources, chunk: int = 64, on_rows=None):
    """The uniform estimate over the given draws (n/k times the exact sums of
    the oracle's rows), computed on all cores. on_rows(i0, rows) sees every
    chunk of oracle rows (for element-wise comparisons) before it is summed."""
    k = len(sources)
    acc = oracle.UniformAccumulator(g.n)
    w = workers()
    try:
        with ThreadPoolExecutor(max_workers=w) as pool:
            for i0 in range(0, k, chunk):
                rows = dependency_rows(g, sources[i0:i0 + chunk], pool)
                if on_rows is not None:
                    on_rows(i0, rows)
                add_rows_parallel(acc, rows, pool, w)
        return acc.estimate(k)
    finally:
        acc.close()


def target_columns(g, sources, targets, chunk: int = 256) -> np.ndarray:
    """delta_{s_i}(v_j) for every draw i and target j: [len(sources)][T]."""
    t = np.asarray(targets, np.int64)
    out = np.empty((len(sources), t.shape[0]), np.float64)
    with ThreadPoolExecutor(max_workers=workers()) as pool:
        for i0 in range(0, len(sources), chunk):
            part = list(pool.map(lambda s: oracle.dependencies(g, int(s))[0][t], sources[i0:i0 + chunk]))
            out[i0:i0 + len(part)] = np.stack(part)
    return out


def pair_values(g, targets, seed: int, qid: int, count: int) -> np.ndarray:
    """y[j][i] for draws 0..count-1 (Algorithm 1), blocks of draws on all cores."""
    w = workers()
    cuts = np.linspace(0, count, w + 1).astype(np.int64)
    blocks = [(int(cuts[i]), int(cuts[i + 1] - cuts[i])) for i in range(w) if cuts[i + 1] > cuts[i]]
    with ThreadPoolExecutor(max_workers=w) as pool:
        parts = list(pool.map(lambda b: oracle.pair_sequence_multi(g, targets, seed, qid, b[0], b[1]), blocks))
    return np.concatenate(parts, axis=1)


def replay_bader(X: np.ndarray, n: int, c: float, cap: int):
    """Sec. 4 steps 2-3 per target over the draw-ordered values X[i][j]:
    S <- S + x_i; k <- i+1; stop at the first S > c*n, or at the cap.
    Returns k, S, status (0 stopped, 1 capped), est = (n*S)/k."""
    T = X.shape[1]
    k = np.zeros(T, np.int64)
    S = np.zeros(T, np.float64)
    st = np.ones(T, np.int32)
    cn = c * n
    for j in range(T):
        s = 0.0
        kk = 0
        for i in range(min(cap, X.shape[0])):
            s = s + float(X[i, j])
            kk = i + 1
            if s > cn:
                st[j] = 0
                break
        k[j], S[j] = kk, s
    est = np.array([(n * S[j]) / k[j] for j in range(T)])
    return k, S, st, est


def replay_pairs(Y: np.ndarray, n: int, c: float, cap: int, scale: float = 1.0):
    """Algorithm 1's loop per target over y[j][i]: S <- S + y_i; k <- i+1; stop
    at the first S*scale > c*n, or at the cap; est = (n(n-1)*S)/k."""
    T = Y.shape[0]
    k = np.zeros(T, np.int64)
    S = np.zeros(T, np.float64)
    st = np.ones(T, np.int32)
    cn = c * n
    for j in range(T):
        s = 0.0
        kk = 0
        for i in range(min(cap, Y.shape[1])):
            s = s + float(Y[j, i])
            kk = i + 1
            if s * scale > cn:
                st[j] = 0
                break
        k[j], S[j] = kk, s
    est = np.array([(n * (n - 1.0) * S[j]) / k[j] for j in range(T)])
    return k, S, st, est
