"""bc_uniform_sources_multi: many graphs of uneven size and depth in one
persistent launch. Each graph's estimate must equal the oracle's uniform
estimate (and the per-graph call) bit for bit, on a mix that exercises hub
vertices (degree > 32, warp-cooperative path), isolated vertices, deep grids
whose corner samples overflow 64-bit counts (extended form), tiny graphs, and
a replay of the captured launch sequence."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _mix():
    path = gg.from_edges(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    single = gg.from_edges(1, np.zeros(0, np.int32), np.zeros(0, np.int32))
    return [
        (gg.erdos_renyi(1500, 6, 11), 100),
        (gg.rmat(11, 8, 0.57, 0.19, 0.19, 12), 130),
        (gg.grid(40), 70),
        (gg.grid(12), 64),
        (gg.barabasi_albert(3000, 3, 13), 37),
        (path, 5),
        (single, 3),
        (gg.erdos_renyi(4000, 16, 14), 1),
    ]


def test_multi_matches_oracle_and_per_graph_calls():
    import paper_1608_04472_gb300 as pkg

    mix = _mix()
    seeds = [100 + i for i in range(len(mix))]
    qids = [7 * i + 1 for i in range(len(mix))]
    with pkg.Context(0, batch_width=64) as ctx:
        hs = [ctx.load_graph(g.row_ptr, g.col) for g, _ in mix]
        ks = [k for _, k in mix]
        first = ctx.uniform_sources_multi(hs, ks, seeds, qids)
        again = ctx.uniform_sources_multi(hs, ks, seeds, qids)  # replay of the captured graph
        single = [ctx.uniform_sources(h, k, s, q) for h, k, s, q in zip(hs, ks, seeds, qids)]
        other = ctx.uniform_sources_multi(hs[:3], [5, 5, 5], seeds[:3], qids[:3])  # a new plan
    for i, (g, k) in enumerate(mix):
        ref = oracle.uniform_sources(g, k, seeds[i], qids[i])
        assert np.array_equal(first[i], ref), (i, np.sum(first[i] != ref))
        assert np.array_equal(again[i], ref), i
        assert np.array_equal(single[i], ref), i
    for i in range(3):
        assert np.array_equal(other[i], oracle.uniform_sources(mix[i][0], 5, seeds[i], qids[i])), i


def test_multi_rejects_bad_arguments():
    import paper_1608_04472_gb300 as pkg

    g = gg.grid(5)
    with pkg.Context(0) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        with pytest.raises(pkg.BCError):
            ctx.uniform_sources_multi([h], [0], [1], [1])
        with pytest.raises(pkg.BCError):
            ctx.uniform_sources_multi([h, 12345], [1, 1], [1, 1], [1, 1])
        # freeing a graph of the cached plan drops the plan; a new call works
        ctx.uniform_sources_multi([h], [4], [1], [1])
        ctx.free_graph(h)
        h2 = ctx.load_graph(g.row_ptr, g.col)
        out = ctx.uniform_sources_multi([h2], [4], [1], [1])
        assert np.array_equal(out[0], oracle.uniform_sources(g, 4, 1, 1))


def test_uneven_set_full_size_sampled():
    """The full uneven workload (256 graphs, 1024 draws each) in one call; the
    two smallest graphs of each family and one deeper grid are checked against
    the oracle."""
    import paper_1608_04472_gb300 as pkg

    S = gg.uneven_set()
    G = len(S)
    seeds = [6000 + i for i in range(G)]
    qids = list(range(G))
    with pkg.Context(0, batch_width=64) as ctx:
        hs = [ctx.load_graph(g.row_ptr, g.col) for _, g in S]
        out = ctx.uniform_sources_multi(hs, [1024] * G, seeds, qids)
    checked = 0
    for fam in ["er", "rmat", "grid"]:
        order = sorted((i for i, (f, _) in enumerate(S) if f == fam), key=lambda i: S[i][1].n)
        idx = order[:2]
        if fam == "grid":  # and one deeper grid (side ~90, ~180 levels)
            idx.append(next(i for i in order if S[i][1].n > 8000))
        for i in idx:
            ref = oracle.uniform_sources(S[i][1], 1024, seeds[i], qids[i])
            assert np.array_equal(out[i], ref), (fam, i, np.sum(out[i] != ref))
            checked += 1
    assert checked == 7
    for i, (_, g) in enumerate(S):
        assert out[i].shape == (g.n,) and np.all(np.isfinite(out[i])) and np.all(out[i] >= 0)
