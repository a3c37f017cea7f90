"""The library's tuner on the GPU: bc_autotune on an R-MAT graph with hubs
keeps only settings whose estimate is bit-identical (checked inside), the
chosen setting stays with the graph (later calls, served queries and the
uniform estimate all equal the oracle), bc_set_tuning / bc_get_tuning round-
trip and reject bad values, and the cache restores a choice in a new context."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results_and_the_choice_stays_with_the_graph(tmp_path):
    import paper_1608_04472_gb300 as pkg
    from paper_1608_04472_gb300 import autotune as at
    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, 91)
    with pkg.Context(0, batch_width=64) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        before = ctx.get_tuning(h)
        t = at.tune_cached(ctx, h, g.row_ptr, g.col, str(tmp_path / "t.json"), k=128, seed=3)
        assert t["cached"] is False and t["trial_ms"] > 0
        now = ctx.get_tuning(h)
        for name in pkg.capi.TUNING_FIELDS:
            assert now[name] == t[name], name
        assert before["batch_width"] == 64
        assert np.array_equal(ctx.uniform_sources(h, 96, 5, 6), oracle.uniform_sources(g, 96, 5, 6))
        tk = ctx.submit(h, pkg.BC_QUERY_SOURCES, targets=[0, 1, 2], c=2.0, cap=400, seed=7, qid=8)
        ctx.poll(tk, -1)
        ref = oracle.adaptive_sources(g, [0, 1, 2], 2.0, 400, 7, 8)
        assert np.array_equal(tk.outputs()["k"], ref["k"]) and np.array_equal(tk.outputs()["est"], ref["est"])
        bad = dict(now)
        bad["batch_width"] = 7
        with pytest.raises(pkg.BCError):
            ctx.set_tuning(h, bad)
        # every knob at a non-default value gives the oracle's results too
        odd = dict(now, heavy_degree=128, segment=128, packed_max_lanes=32, packed_min_preds=4, bwd_variant=0,
                   heavy_lane=1, push_div=1000)
        ctx.set_tuning(h, odd)
        assert np.array_equal(ctx.uniform_sources(h, 96, 5, 6), oracle.uniform_sources(g, 96, 5, 6))
    with pkg.Context(0, batch_width=64) as ctx2:
        h2 = ctx2.load_graph(g.row_ptr, g.col)
        t2 = at.tune_cached(ctx2, h2, g.row_ptr, g.col, str(tmp_path / "t.json"))
        assert t2["cached"] is True
        assert all(ctx2.get_tuning(h2)[k] == t[k] for k in pkg.capi.TUNING_FIELDS)
