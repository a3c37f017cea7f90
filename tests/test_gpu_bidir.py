"""GPU parity of pair sampling (Algorithm 1) through the bidirectional pair
search: d(s,t) and sigma_st from two balls meeting in the middle must give
estimates, draw counts, sums and stop states equal to the oracle's bit for bit.
Cases: a small-world graph over windows of up to 1024 draws; an R-MAT graph
whose hubs are expanded by whole CTAs; a sparse graph
with many unreachable pairs and isolated vertices; tiny graphs (adjacent
pairs); a 90x90 grid where many sigma_st exceed 2^64 (extended form) and others
lie below 2^64 while counts elsewhere at the same depth do not (R11 for pairs).
The one-sided engine (BCG_PAIR_ENGINE=1), the one-pair-per-warp search
(BCG_PAIR_ENGINE=2), the plain width and the served query must agree too, and
so must the one-pair-per-warp search when small tables (BCG_PAIR_HASH) make it
hand most pairs, or some of them, to the CTA search."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

KEYS = ["est", "k", "S", "status"]


@pytest.fixture(scope="module")
def pkg():
    import paper_1608_04472_gb300 as p
    return p


def _run(pkg, g, targets, c, cap, seed, qid, width=64, scale=1.0, served=False):
    with pkg.Context(0, batch_width=width) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        out = ctx.adaptive_pairs(h, targets, c, cap, seed, qid, scale)
        if served:
            tk = ctx.submit(h, pkg.BC_QUERY_PAIRS, targets=targets, c=c, cap=cap, seed=seed, qid=qid,
                            threshold_scale=scale)
            assert ctx.poll(tk, -1) == pkg.BC_OK
            return out, tk.outputs()
    return out, None


def _same(got, ref, what):
    for key in KEYS:
        assert np.array_equal(got[key], ref[key]), (what, key, got[key][:8], ref[key][:8])


@pytest.mark.parametrize("engine", ["0", "1", "2"])
def test_small_world_windows(pkg, monkeypatch, engine):
    monkeypatch.setenv("BCG_PAIR_ENGINE", engine)
    g = gg.barabasi_albert(20000, 4, 41)
    targets = gg.degree_targets(g, 16, 42)
    ref = oracle.adaptive_pairs(g, targets, 1.0, 3000, 4, 7)
    got, served = _run(pkg, g, targets, 1.0, 3000, 4, 7, served=True)
    _same(got, ref, "batched")
    _same(served, ref, "served")
    assert np.all(ref["k"] == 3000)  # every target ran through windows of up to 1024 draws


@pytest.mark.parametrize("engine", ["0", "2"])
def test_hub_vertices_expanded_by_the_whole_cta(pkg, monkeypatch, engine):
    # R-MAT s13 has 27 vertices of degree above 512 (up to 2,204): frontiers
    # holding them are expanded by all threads of the CTA (engine 0) or by the
    # whole warp (engine 2)
    monkeypatch.setenv("BCG_PAIR_ENGINE", engine)
    g = gg.rmat(13, 16, 0.57, 0.19, 0.19, 46)
    assert int(np.diff(g.row_ptr).max()) > 2000
    targets = gg.degree_targets(g, 12, 47)
    ref = oracle.adaptive_pairs(g, targets, 1.0, 2500, 11, 3)
    got, served = _run(pkg, g, targets, 1.0, 2500, 11, 3, served=True)
    _same(got, ref, "batched")
    _same(served, ref, "served")


def test_small_world_stops_and_plain_width(pkg):
    g = gg.barabasi_albert(3000, 3, 43)
    targets = gg.degree_targets(g, 12, 44)
    scale = float(g.n - 1)
    ref = oracle.adaptive_pairs(g, targets, 2.0, 5000, 6, 8, scale)
    assert np.any(ref["status"] == 0) and np.any(ref["k"] > 64)
    got, _ = _run(pkg, g, targets, 2.0, 5000, 6, 8, scale=scale)
    _same(got, ref, "batched")
    ref1 = oracle.adaptive_pairs(g, targets, 2.0, 150, 6, 8, scale)
    got1, _ = _run(pkg, g, targets, 2.0, 150, 6, 8, width=1, scale=scale)
    _same(got1, ref1, "plain")


def test_unreachable_pairs_and_isolated_vertices(pkg):
    g = gg.erdos_renyi(3000, 1.2, 45)  # below the giant-component threshold in part: many components
    deg = np.diff(g.row_ptr)
    assert np.sum(deg == 0) > 100
    targets = [int(v) for v in np.argsort(-deg)[:10]] + [int(np.argmin(deg))]
    ref = oracle.adaptive_pairs(g, targets, 1.0, 2500, 9, 2)
    got, served = _run(pkg, g, targets, 1.0, 2500, 9, 2, served=True)
    _same(got, ref, "batched")
    _same(served, ref, "served")


@pytest.mark.parametrize("make", [
    lambda: gg.from_edges(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32)),
    lambda: gg.from_edges(6, np.zeros(5, np.int32), np.arange(1, 6, dtype=np.int32)),
    lambda: gg.from_edges(2, np.array([0], np.int32), np.array([1], np.int32)),
])
def test_tiny_graphs(pkg, make):
    g = make()
    targets = list(range(g.n))
    ref = oracle.adaptive_pairs(g, targets, 1.0, 300, 3, 3)
    got, _ = _run(pkg, g, targets, 1.0, 300, 3, 3)
    _same(got, ref, "tiny")


@pytest.mark.parametrize("engine,width", [("0", 64), ("1", 64), ("2", 64), ("0", 1)])
def test_grid_with_counts_beyond_2_to_64(pkg, monkeypatch, engine, width):
    # about 3 in 10 draws have sigma_st >= 2^64 (extended form); about 1 in 10
    # have sigma_st < 2^64 while other counts at depth <= d(s,t) from s exceed
    # it, where sigma_st is the exact count (R11 for pairs)
    monkeypatch.setenv("BCG_PAIR_ENGINE", engine)
    g = gg.grid(90)
    targets = [45 * 90 + 45, 30 * 90 + 70, 60 * 90 + 20, 20 * 90 + 30, 70 * 90 + 60, 0]
    cap = 400 if width == 64 else 60
    ref = oracle.adaptive_pairs(g, targets, 1.0, cap, 5, 9)
    got, _ = _run(pkg, g, targets, 1.0, cap, 5, 9, width=width)
    _same(got, ref, f"engine {engine} width {width}")
    assert np.sum(ref["S"] > 0) >= 5


@pytest.mark.parametrize("lg", ["6", "9"])
def test_warp_search_hands_large_balls_to_the_cta_search(pkg, monkeypatch, lg):
    # 2^6 slots per side: nearly every pair outgrows its table (32 vertices);
    # 2^9: some do. Either way the results are the oracle's.
    monkeypatch.setenv("BCG_PAIR_ENGINE", "2")
    monkeypatch.setenv("BCG_PAIR_HASH", lg)
    g = gg.barabasi_albert(20000, 4, 41)
    targets = gg.degree_targets(g, 16, 42)
    ref = oracle.adaptive_pairs(g, targets, 1.0, 2000, 4, 9)
    with pkg.Context(0, batch_width=64) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        ctx.reset_stats()
        got = ctx.adaptive_pairs(h, targets, 1.0, 2000, 4, 9)
        fb = ctx.stats()["pair_fallbacks"]
    _same(got, ref, f"hash 2^{lg}")
    assert fb > (1000 if lg == "6" else 0), fb
