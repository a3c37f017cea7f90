"""The autotuner on the GPU: trials over a small grid on an R-MAT graph give
bit-identical estimates (checked inside tune), and a context made with the
chosen settings matches the oracle."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def test_tune_small_grid_and_use_the_result(tmp_path):
    from paper_1608_04472_gb300 import autotune as at
    g = gg.rmat(12, 8, 0.57, 0.19, 0.19, 91)
    grid = {"BCG_HEAVY_DEGREE": (256, 128), "BCG_BWD_VARIANT": (1, 0), "BCG_PK_MINCNT": (6, 4)}
    res = at.tune_cached(g.row_ptr, g.col, str(tmp_path / "t.json"), grid=grid, k=128)
    assert set(res["best"]) == set(grid) and res["seconds"] > 0
    for name, v in res["best"].items():
        assert v in grid[name]
    ctx = at.tuned_context(res["best"])
    try:
        h = ctx.load_graph(g.row_ptr, g.col)
        got = ctx.uniform_sources(h, 96, 5, 6)
    finally:
        ctx.close()
    assert np.array_equal(got, oracle.uniform_sources(g, 96, 5, 6))
