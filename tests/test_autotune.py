"""Host logic of the autotuner (no GPU): coordinate descent from the defaults
over a fake timing function, the check that knobs never change a result, the
per-graph cache and the environment it sets while a context is created."""
import os

import numpy as np
import pytest

import graphgen as gg
from paper_1608_04472_gb300 import autotune as at


def _fake(times, est=None, log=None):
    est = np.arange(5.0) if est is None else est

    def runner(s):
        if log is not None:
            log.append(dict(s))
        return times(s), est
    return runner


def test_coordinate_descent_picks_the_fastest_value_per_knob():
    grid = {"A": (1, 2, 3), "B": (10, 20)}
    # A = 2 is fastest; with A = 2, B = 20 is fastest
    cost = lambda s: {1: 5.0, 2: 1.0, 3: 4.0}[s["A"]] + (0.5 if s["B"] == 10 else 0.1)
    log = []
    res = at.tune(None, None, grid=grid, runner=_fake(cost, log=log))
    assert res["best"] == {"A": 2, "B": 20}
    assert res["seconds"] == pytest.approx(1.1)
    # defaults first, shared setting not rerun: 3 + 2 - 1 trials
    assert log[0] == {"A": 1, "B": 10} and len(log) == 4 and len(res["trials"]) == 4


def test_ties_keep_the_smaller_value():
    res = at.tune(None, None, grid={"A": (3, 1, 2)}, runner=_fake(lambda s: 1.0))
    assert res["best"] == {"A": 1}


def test_a_knob_that_changes_a_result_is_refused():
    calls = []

    def runner(s):
        calls.append(s)
        return 1.0, np.array([1.0, 2.0 if s["A"] == 1 else 2.0000000000000004])

    with pytest.raises(AssertionError):
        at.tune(None, None, grid={"A": (1, 2)}, runner=runner)


def test_empty_grid_entry_is_an_error():
    with pytest.raises(ValueError):
        at.tune(None, None, grid={"A": ()}, runner=_fake(lambda s: 1.0))


def test_cache_runs_once_per_graph(tmp_path):
    g = gg.erdos_renyi(300, 4, 3)
    h = gg.erdos_renyi(300, 4, 4)
    path = str(tmp_path / "tune.json")
    log = []
    kw = dict(grid={"A": (1, 2)}, runner=_fake(lambda s: float(s["A"]), log=log))
    r1 = at.tune_cached(g.row_ptr, g.col, path, **kw)
    r2 = at.tune_cached(g.row_ptr, g.col, path, **kw)
    assert r1 == r2 == {"best": {"A": 1}, "seconds": 1.0} and len(log) == 2
    at.tune_cached(h.row_ptr, h.col, path, **kw)
    assert len(log) == 4 and len(at.load_cache(path)) == 2


def test_signature_depends_on_the_arrays():
    g = gg.erdos_renyi(300, 4, 3)
    col = g.col.copy()
    col[0] = col[1]
    assert at.graph_signature(g.row_ptr, g.col) == at.graph_signature(g.row_ptr.copy(), g.col.copy())
    assert at.graph_signature(g.row_ptr, g.col) != at.graph_signature(g.row_ptr, col)


def test_defaults_come_first_and_the_environment_is_restored(monkeypatch):
    for name, values in at.DEFAULT_GRID.items():
        assert len(values) >= 2 and len(set(values)) == len(values), name
    monkeypatch.setenv("BCG_SEGMENT", "999")
    monkeypatch.delenv("BCG_HEAVY_DEGREE", raising=False)
    with at._Env({"BCG_SEGMENT": 512, "BCG_HEAVY_DEGREE": 128}):
        assert os.environ["BCG_SEGMENT"] == "512" and os.environ["BCG_HEAVY_DEGREE"] == "128"
    assert os.environ["BCG_SEGMENT"] == "999" and "BCG_HEAVY_DEGREE" not in os.environ
