"""Host side of the tuner (no GPU): the cache across processes, the graph
signature, and the binding's copy of the bc_tuning struct against the header
(field names, order and types)."""
import os
import re

import pytest

import graphgen as gg
from paper_1608_04472_gb300 import autotune as at

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bc.h")


class _FakeCtx:
    """Records the calls tune_cached makes."""

    def __init__(self):
        self.calls = []

    def autotune(self, g, k, seed):
        self.calls.append(("autotune", g, k, seed))
        return {"batch_width": 64, "heavy_degree": 512, "segment": 256, "packed_max_lanes": 16,
                "packed_min_preds": 6, "bwd_variant": 1, "heavy_lane": 0, "push_div": 32, "deep_levels": 32,
                "trial_ms": 3.5}

    def set_tuning(self, g, t):
        self.calls.append(("set", g, dict(t)))


def test_cache_tunes_once_per_graph_and_restores_after(tmp_path):
    g = gg.erdos_renyi(300, 4, 3)
    h = gg.erdos_renyi(300, 4, 4)
    path = str(tmp_path / "tune.json")
    c1 = _FakeCtx()
    r1 = at.tune_cached(c1, 7, g.row_ptr, g.col, path, k=64, seed=2)
    assert r1["cached"] is False and c1.calls == [("autotune", 7, 64, 2)]
    c2 = _FakeCtx()  # another process: restored, not tuned
    r2 = at.tune_cached(c2, 9, g.row_ptr, g.col, path)
    assert r2["cached"] is True and c2.calls[0][0] == "set" and c2.calls[0][1] == 9
    assert c2.calls[0][2]["heavy_degree"] == 512 and len(c2.calls) == 1
    at.tune_cached(c2, 10, h.row_ptr, h.col, path)
    assert c2.calls[-1][0] == "autotune" and len(at.load_cache(path)) == 2


def test_signature_depends_on_the_arrays():
    g = gg.erdos_renyi(300, 4, 3)
    col = g.col.copy()
    col[0] = col[1]
    assert at.graph_signature(g.row_ptr, g.col) == at.graph_signature(g.row_ptr.copy(), g.col.copy())
    assert at.graph_signature(g.row_ptr, g.col) != at.graph_signature(g.row_ptr, col)


def test_binding_struct_matches_the_header():
    from paper_1608_04472_gb300 import capi
    text = open(HEADER).read()
    body = re.search(r"typedef struct bc_tuning \{(.*?)\} bc_tuning;", text, re.S).group(1)
    fields = re.findall(r"^\s*(int32_t|double)\s+(\w+);", body, re.M)
    declared = [(name, ty) for ty, name in fields]
    bound = [(name, "double" if t.__name__ == "c_double" else "int32_t") for name, t in capi.bc_tuning._fields_]
    assert declared == bound
    assert set(capi.TUNING_FIELDS) == {n for n, _ in declared} - {"reserved0", "trial_ms"}
