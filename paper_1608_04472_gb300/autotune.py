"""Autotuner for the batched engine's launch knobs.

The library reads its tuning knobs when a context is created (environment
variables ``BCG_*``): the degree above which a vertex is split into segments
(warp vs segment expansion), the segment length, the packed-chunk threshold of
the forward pass, the backward kernel form and the depth above which a graph
runs lane-major (level masks vs one source per CTA). Defaults come from sweeps
on one R-MAT graph; this module picks them per graph by timing a short uniform
estimate (the per-sample step of Sec. 3 summed over k draws) under each
setting, one knob at a time (coordinate descent from the defaults).

Every sum that decides a result is exact, so the knobs may change the speed
but never an output bit: each trial's estimate is compared with the first one
and a difference raises. Results are cached per graph signature in a JSON
file, and ``tuned_context`` makes a context with the chosen settings.
"""
from __future__ import annotations

import hashlib
import json
import os
import time
from typing import Callable

import numpy as np

# knob -> values tried, the first being the library default
DEFAULT_GRID: dict[str, tuple[int, ...]] = {
    "BCG_HEAVY_DEGREE": (256, 128, 512),
    "BCG_SEGMENT": (256, 512),
    "BCG_PK_MINCNT": (6, 4, 8),
    "BCG_BWD_VARIANT": (1, 0),
    "BCG_DEEP_LEVELS": (32, 16, 64),
}


def graph_signature(row_ptr, col) -> str:
    """A stable key for a CSR graph (its size and a hash of both arrays)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    h = hashlib.sha256()
    h.update(np.array([rp.shape[0] - 1, cl.shape[0]], np.int64).tobytes())
    h.update(rp.tobytes())
    h.update(cl.tobytes())
    return h.hexdigest()[:32]


class _Env:
    """Sets BCG_* variables for the duration of a context creation."""

    def __init__(self, settings: dict[str, int]):
        self.settings = settings
        self.saved: dict[str, str | None] = {}

    def __enter__(self):
        for k, v in self.settings.items():
            self.saved[k] = os.environ.get(k)
            os.environ[k] = str(int(v))
        return self

    def __exit__(self, *exc):
        for k, v in self.saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def tuned_context(settings: dict[str, int], device: int = 0, batch_width: int = 64, stream=None):
    """A Context whose knobs are `settings` (read once, at creation)."""
    from . import capi
    with _Env(settings):
        return capi.Context(device, batch_width, stream)


def gpu_trial(row_ptr, col, settings: dict[str, int], k: int = 256, seed: int = 1, qid: int = 0,
              device: int = 0) -> tuple[float, np.ndarray]:
    """Seconds of one uniform k-draw estimate under `settings` (after a warm-up
    call that builds the per-graph metadata), and the estimate."""
    ctx = tuned_context(settings, device)
    try:
        h = ctx.load_graph(row_ptr, col)
        ctx.uniform_sources(h, max(1, k // 4), seed, qid + 1)
        t0 = time.perf_counter()
        est = ctx.uniform_sources(h, k, seed, qid)
        return time.perf_counter() - t0, est
    finally:
        ctx.close()


def tune(row_ptr, col, grid: dict[str, tuple[int, ...]] | None = None,
         runner: Callable[[dict[str, int]], tuple[float, np.ndarray]] | None = None, k: int = 256,
         device: int = 0) -> dict:
    """Coordinate descent over `grid` from its first values. `runner(settings)`
    returns (seconds, estimate); by default a GPU trial of a uniform k-draw
    estimate. Returns {"best": settings, "seconds": time of the best,
    "trials": [(settings, seconds), ...]}. Raises AssertionError when two
    settings give different estimates."""
    grid = dict(grid or DEFAULT_GRID)
    for name, values in grid.items():
        if not values:
            raise ValueError(f"no values for {name}")
    if runner is None:
        def runner(settings):
            return gpu_trial(row_ptr, col, settings, k=k, device=device)
    best = {name: int(values[0]) for name, values in grid.items()}
    seen: dict[tuple, float] = {}
    trials: list[tuple[dict[str, int], float]] = []
    ref = None

    def run(settings):
        nonlocal ref
        key = tuple(sorted(settings.items()))
        if key in seen:
            return seen[key]
        t, est = runner(dict(settings))
        est = np.asarray(est)
        if ref is None:
            ref = est
        elif not np.array_equal(est, ref):
            raise AssertionError(f"estimate changed under {settings}: the knobs must not change results")
        seen[key] = float(t)
        trials.append((dict(settings), float(t)))
        return float(t)

    for name, values in grid.items():
        timed = []
        for v in values:
            s = dict(best)
            s[name] = int(v)
            timed.append((run(s), int(v)))
        best[name] = min(timed)[1]  # ties keep the smaller value
    return {"best": best, "seconds": seen[tuple(sorted(best.items()))], "trials": trials}


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except FileNotFoundError:
        return {}


def tune_cached(row_ptr, col, path: str, **kw) -> dict:
    """`tune` once per graph signature; later calls read the JSON cache."""
    sig = graph_signature(row_ptr, col)
    cache = load_cache(path)
    if sig in cache:
        return cache[sig]
    res = tune(row_ptr, col, **kw)
    cache[sig] = {"best": res["best"], "seconds": res["seconds"]}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return cache[sig]
