"""BC_NORMALIZE at load: rows sorted, self-loops and duplicate columns dropped
(a duplicate edge with lengths keeps the shortest), so a messy CSR of a graph
gives the same results as the clean CSR of that graph, and the stored nnz is
the clean count."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _messy(g, rng, lengths=None):
    """Each row shuffled, with self-loops and repeated entries added; repeated
    entries get longer lengths than the original so the shortest is kept."""
    rows, wrows = [], []
    for v in range(g.n):
        a, b = g.row_ptr[v], g.row_ptr[v + 1]
        cols = list(g.col[a:b])
        ws = list(lengths[a:b]) if lengths is not None else [1] * (b - a)
        extra = [int(c) for c in rng.choice(cols, size=min(len(cols), 2), replace=False)] if cols else []
        cols2 = cols + extra + ([v] if v % 3 == 0 else [])
        ws2 = ws + [int(ws[cols.index(c)]) + 5 for c in extra] + ([7] if v % 3 == 0 else [])
        perm = rng.permutation(len(cols2))
        rows.append([cols2[i] for i in perm])
        wrows.append([ws2[i] for i in perm])
    rp = np.zeros(g.n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c in r], np.int32)
    w = np.array([x for r in wrows for x in r], np.uint32)
    return rp, col, w


def test_normalize_gives_the_clean_graph():
    import paper_1608_04472_gb300 as pkg
    rng = np.random.default_rng(5)
    g = gg.erdos_renyi(800, 6, 2)
    rp, col, _ = _messy(g, rng)
    srcs = [0, 17, 799]
    with pkg.Context(0, batch_width=64) as ctx:
        with pytest.raises(pkg.BCError):
            ctx.load_graph(rp, col, validate=True)  # loops, duplicates, unsorted rows
        h = ctx.load_graph(rp, col, validate=True, normalize=True)
        assert pkg.capi.bc_graph_info(ctx.ptr, h) == (g.n, g.nnz)
        delta, _, _ = ctx.source_dependencies(h, srcs)
        res = ctx.adaptive_sources(h, [1, 2, 3], 2.0, 300, 4, 5)
    for i, s in enumerate(srcs):
        assert np.array_equal(delta[i], oracle.dependencies(g, s)[0])
    ref = oracle.adaptive_sources(g, [1, 2, 3], 2.0, 300, 4, 5)
    assert np.array_equal(res["k"], ref["k"]) and np.array_equal(res["est"], ref["est"])


def test_normalize_keeps_the_shortest_duplicate_length():
    import paper_1608_04472_gb300 as pkg
    rng = np.random.default_rng(6)
    g = gg.erdos_renyi(500, 5, 3)
    wl = gg.edge_lengths(g, 1, 20, 4)
    rp, col, w = _messy(g, rng, wl)
    with pkg.Context(0, batch_width=64) as ctx:
        h = ctx.load_graph(rp, col, validate=True, lengths=w, normalize=True)
        d, dist, _, _, _, _ = ctx.source_dependencies_weighted(h, [0, 250])
    for i, s in enumerate([0, 250]):
        d_o, dist_o, _, _, _, _ = oracle.dependencies_w(g, wl, s)
        assert np.array_equal(d[i], d_o) and np.array_equal(dist[i], dist_o)
