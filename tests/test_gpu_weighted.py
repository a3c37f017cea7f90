"""GPU parity on weighted graphs (positive integer edge lengths; Sec. 3 step 1
with Dijkstra, Def. 3 with lengths, Theorem 1): the weighted engine's
per-source rows (int64 distances, counts, dependencies, including samples
beyond 2^64 in the extended form), exact BC, the uniform estimate, Bader's
sampling (called and served) and the multi-graph call must equal the oracle
bit for bit; graphs without lengths through the weighted engine must equal the
unweighted engines."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1608_04472_gb300 as p
    return p


def _cases():
    er = gg.erdos_renyi(2000, 6, 71)
    rm = gg.rmat(11, 8, 0.57, 0.19, 0.19, 72)  # hubs: warp-wide rows
    ba = gg.barabasi_albert(3000, 3, 73)
    dr = gg.directed_rmat(10, 8, 0.57, 0.19, 0.19, 74)
    return {
        "er_1_100": (er, gg.edge_lengths(er, 1, 100, 75), False),
        "rmat_1_4": (rm, gg.edge_lengths(rm, 1, 4, 76), False),  # many ties: counts > 1
        "ba_1_1000": (ba, gg.edge_lengths(ba, 1, 1000, 77), False),
        "directed_rmat_1_8": (dr, gg.edge_lengths(dr, 1, 8, 78, symmetric=False), True),
    }


@pytest.mark.parametrize("name", ["er_1_100", "rmat_1_4", "ba_1_1000", "directed_rmat_1_8"])
def test_weighted_source_rows(pkg, name):
    g, w, directed = _cases()[name]
    rng = np.random.default_rng(9)
    sources = [0, g.n - 1] + rng.integers(0, g.n, 80).tolist()
    with pkg.Context(0, batch_width=64) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col, validate=True, directed=directed, lengths=w)
        delta, dist, sig, sm, se, tier = ctx.source_dependencies_weighted(h, sources)
        d2, sig2 = ctx.source_dependencies(h, sources, want_sigma=True)[0::2]
    for i, s in enumerate(sources):
        ed, edist, esig, ovf, esm, ese = oracle.dependencies_w(g, w, s)
        assert tier[i] == int(ovf), (i, s)
        assert np.array_equal(dist[i], edist), (i, s)
        assert np.array_equal(sig[i], esig), (i, s)
        assert np.array_equal(sm[i], esm) and np.array_equal(se[i].astype(np.int64), ese), (i, s)
        assert np.array_equal(delta[i], ed), (i, s, np.sum(delta[i] != ed))
        assert np.array_equal(d2[i], ed) and np.array_equal(sig2[i], esig), (i, s)


def test_equal_lengths_grid_beyond_2_to_64(pkg):
    g = gg.grid(45)
    w = np.full(g.col.shape[0], 3, np.uint32)
    sources = [0, 44, g.n - 1, 22 * 45 + 22, 1, 46]
    with pkg.Context(0, batch_width=64) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col, lengths=w)
        delta, dist, sig, sm, se, tier = ctx.source_dependencies_weighted(h, sources)
    assert tier[0] == 1 and tier[3] == 0
    for i, s in enumerate(sources):
        ed, edist, esig, ovf, esm, ese = oracle.dependencies_w(g, w, s)
        assert tier[i] == int(ovf)
        assert np.array_equal(dist[i], edist) and np.array_equal(sig[i], esig)
        assert np.array_equal(sm[i], esm) and np.array_equal(se[i].astype(np.int64), ese), i
        assert np.array_equal(delta[i], ed), (i, np.sum(delta[i] != ed))


@pytest.mark.parametrize("make", [lambda: gg.rmat(11, 8, 0.57, 0.19, 0.19, 79), lambda: gg.grid(40)])
def test_unit_lengths_through_the_weighted_engine(pkg, make):
    g = make()
    sources = [0, 1, g.n // 2, g.n - 1, 7, 300]
    with pkg.Context(0, batch_width=64) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        delta, dist, sig, sm, se, tier = ctx.source_dependencies_weighted(h, sources)
        d2, dist2, sig2 = ctx.source_dependencies(h, sources, want_dist=True, want_sigma=True)
    assert np.array_equal(delta, d2)
    assert np.array_equal(dist, dist2.astype(np.int64))
    assert np.array_equal(sig, sig2)
    for i, s in enumerate(sources):
        assert np.array_equal(delta[i], oracle.dependencies(g, s)[0]), i


@pytest.mark.parametrize("width", [1, 64])
def test_weighted_exact_bc(pkg, width):
    g = gg.erdos_renyi(300, 5, 80)
    w = gg.edge_lengths(g, 1, 6, 81)
    ref = oracle.exact_bc_w(g, w)
    with pkg.Context(0, batch_width=width) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col, lengths=w)
        got = ctx.exact(h)
    assert np.array_equal(got, ref), np.sum(got != ref)


def test_weighted_uniform_bader_served_and_multi(pkg):
    rm = gg.rmat(11, 8, 0.57, 0.19, 0.19, 82)
    wr = gg.edge_lengths(rm, 1, 20, 83)
    gr = gg.grid(30)
    wg = gg.edge_lengths(gr, 1, 3, 84)
    und = gg.erdos_renyi(1500, 6, 85)
    targets = gg.uniform_targets(rm.n, 10, 86)
    with pkg.Context(0, batch_width=64) as ctx:
        h = ctx.load_graph(rm.row_ptr, rm.col, lengths=wr)
        hg = ctx.load_graph(gr.row_ptr, gr.col, lengths=wg)
        hu = ctx.load_graph(und.row_ptr, und.col)
        got_u = ctx.uniform_sources(h, 300, 5, 2)
        got_b = ctx.adaptive_sources(h, targets, 2.0, 600, 8, 3)
        tk = ctx.submit(h, pkg.BC_QUERY_SOURCES, targets=targets, c=2.0, cap=600, seed=8, qid=3)
        assert ctx.poll(tk, -1) == pkg.BC_OK
        served = tk.outputs()
        multi = ctx.uniform_sources_multi([h, hu, hg], [90, 70, 64], [11, 12, 13], [1, 2, 3])
    assert np.array_equal(got_u, oracle.uniform_sources_w(rm, wr, 300, 5, 2))
    ref_b = oracle.adaptive_sources_w(rm, wr, targets, 2.0, 600, 8, 3)
    for key in ["est", "k", "S", "status"]:
        assert np.array_equal(got_b[key], ref_b[key]), key
        assert np.array_equal(served[key], ref_b[key]), key
    assert np.array_equal(multi[0], oracle.uniform_sources_w(rm, wr, 90, 11, 1))
    assert np.array_equal(multi[1], oracle.uniform_sources(und, 70, 12, 2))
    assert np.array_equal(multi[2], oracle.uniform_sources_w(gr, wg, 64, 13, 3))


def test_weighted_refusals(pkg):
    g = gg.erdos_renyi(200, 4, 87)
    w = gg.edge_lengths(g, 1, 9, 88)
    with pkg.Context(0) as ctx:
        bad = w.copy()
        bad[3] = 0
        with pytest.raises(pkg.BCError):  # lengths must be >= 1
            ctx.load_graph(g.row_ptr, g.col, lengths=bad)
        asym = w.copy()
        asym[0] += 1  # one row of an edge differs from the other
        with pytest.raises(pkg.BCError):
            ctx.load_graph(g.row_ptr, g.col, validate=True, lengths=asym)
        h = ctx.load_graph(g.row_ptr, g.col, validate=True, lengths=w)
        with pytest.raises(pkg.BCError):  # int32 distances: use the weighted entry
            ctx.source_dependencies(h, [1], want_dist=True)
        with pytest.raises(pkg.BCError):
            ctx.adaptive_pairs(h, [1, 2], 1.0, 100, 1, 1)
        with pytest.raises(pkg.BCError):
            ctx.submit(h, pkg.BC_QUERY_PAIRS, targets=[1, 2], c=1.0, cap=100, seed=1, qid=1)
        d = ctx.source_dependencies(h, [5])[0]
        assert np.array_equal(d[0], oracle.dependencies_w(g, w, 5)[0])
