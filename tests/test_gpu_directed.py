"""GPU parity on directed graphs (BC_DIRECTED: paths follow the edges'
direction, BC over ordered pairs, Def. 1). Path counts are pulled over the
in-neighbour CSR the library builds at load; every result must equal the
oracle bit for bit: per-source rows (including corner sources of a directed
grid whose counts exceed 2^64, in the extended form), exact BC, the uniform
estimate, Bader's adaptive sampling (called and served), and the multi-graph
call on a mix of directed and undirected graphs. Pair sampling on a directed
graph is refused."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1608_04472_gb300 as p
    return p


def _graphs():
    return {
        "er": gg.directed_er(2000, 4, 31),
        "rmat": gg.directed_rmat(11, 8, 0.57, 0.19, 0.19, 32),  # in-degrees above 32: warp-wide pulls
        "grid": gg.directed_grid(24),  # most vertices unreachable from most sources
    }


@pytest.mark.parametrize("width", [1, 64])
@pytest.mark.parametrize("name", ["er", "rmat", "grid"])
def test_directed_source_rows(pkg, width, name):
    g = _graphs()[name]
    rng = np.random.default_rng(7)
    sources = [0, g.n - 1] + rng.integers(0, g.n, 70).tolist()
    with pkg.Context(0, batch_width=width) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col, validate=True, directed=True)
        delta, dist, sig = ctx.source_dependencies(h, sources, want_dist=True, want_sigma=True)
    for i, s in enumerate(sources):
        ed, edist, esig, ovf = oracle.dependencies(g, s)
        assert not ovf
        assert np.array_equal(dist[i], edist), (i, s)
        assert np.array_equal(sig[i], esig), (i, s)
        assert np.array_equal(delta[i], ed), (i, s, np.sum(delta[i] != ed))


@pytest.mark.parametrize("width", [1, 64])
def test_directed_grid_extended_rows(pkg, width):
    # from corner 0 of a 45x45 directed grid the count at the far corner is
    # C(88, 44) > 2^64: that source runs in the extended form, pulled over
    # in-neighbours; sources further in stay below 2^64
    g = gg.directed_grid(45)
    sources = [0, 1, 45, 46, 20 * 45 + 20, g.n - 1]
    with pkg.Context(0, batch_width=width) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col, directed=True)
        delta, dist, sm, se, tier = ctx.source_dependencies_ext(h, sources)
    tiers = []
    for i, s in enumerate(sources):
        ed, edist, esig, ovf = oracle.dependencies(g, s)
        tiers.append(int(ovf))
        if ovf:
            _, _, esm, ese = oracle.dependencies_xf(g, s)
            assert np.array_equal(sm[i], esm), (i, s)
            assert np.array_equal(se[i].astype(np.int64), ese), (i, s)
        assert np.array_equal(dist[i], edist), (i, s)
        assert np.array_equal(delta[i], ed), (i, s, np.sum(delta[i] != ed))
    assert tiers[0] == 1 and tiers[-1] == 0
    assert list(tier) == tiers


@pytest.mark.parametrize("width", [1, 64])
def test_directed_exact_bc(pkg, width):
    g = gg.directed_er(400, 3, 33)
    ref = oracle.exact_bc(g)
    with pkg.Context(0, batch_width=width) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col, directed=True)
        got = ctx.exact(h)
    assert np.array_equal(got, ref), np.sum(got != ref)


def test_directed_uniform_and_bader(pkg):
    gs = _graphs()
    with pkg.Context(0, batch_width=64) as ctx:
        for name in ["rmat", "grid"]:
            g = gs[name]
            h = ctx.load_graph(g.row_ptr, g.col, directed=True)
            ref_u = oracle.uniform_sources(g, 300, 5, 2)
            got_u = ctx.uniform_sources(h, 300, 5, 2)
            assert np.array_equal(got_u, ref_u), (name, np.sum(got_u != ref_u))
            targets = gg.uniform_targets(g.n, 10, 4)
            ref_b = oracle.adaptive_sources(g, targets, 2.0, 600, 8, 3)
            got_b = ctx.adaptive_sources(h, targets, 2.0, 600, 8, 3)
            tk = ctx.submit(h, pkg.BC_QUERY_SOURCES, targets=targets, c=2.0, cap=600, seed=8, qid=3)
            assert ctx.poll(tk, -1) == pkg.BC_OK
            served = tk.outputs()
            for key in ["est", "k", "S", "status"]:
                assert np.array_equal(got_b[key], ref_b[key]), (name, key)
                assert np.array_equal(served[key], ref_b[key]), (name, key)


@pytest.mark.parametrize("width", [1, 64])
def test_directed_uniform_with_extended_sources(pkg, width):
    # about a tenth of the 45x45 directed grid's vertices are sources whose
    # counts exceed 2^64 (lane-major: counts recomputed in the extended form)
    g = gg.directed_grid(45)
    k = 200 if width == 64 else 40
    ref = oracle.uniform_sources(g, k, 21, 6)
    with pkg.Context(0, batch_width=width) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col, directed=True)
        got = ctx.uniform_sources(h, k, 21, 6)
    assert np.array_equal(got, ref), np.sum(got != ref)


def test_directed_multi_graph_mix(pkg):
    gs = _graphs()
    und = gg.erdos_renyi(1500, 6, 34)
    mix = [(gs["er"], True), (und, False), (gs["rmat"], True), (gs["grid"], True)]
    ks, seeds, qids = [90, 70, 130, 64], [11, 12, 13, 14], [1, 2, 3, 4]
    with pkg.Context(0, batch_width=64) as ctx:
        hs = [ctx.load_graph(g.row_ptr, g.col, directed=d) for g, d in mix]
        out = ctx.uniform_sources_multi(hs, ks, seeds, qids)
    for i, (g, _) in enumerate(mix):
        ref = oracle.uniform_sources(g, ks[i], seeds[i], qids[i])
        assert np.array_equal(out[i], ref), (i, np.sum(out[i] != ref))


def test_directed_load_flags_and_pair_refusal(pkg):
    g = gg.directed_er(200, 3, 35)
    with pkg.Context(0) as ctx:
        with pytest.raises(pkg.BCError):  # neither flag
            pkg.capi.bc_graph_load_csr(ctx.ptr, g.row_ptr, g.col, 0)
        with pytest.raises(pkg.BCError):  # both flags
            pkg.capi.bc_graph_load_csr(ctx.ptr, g.row_ptr, g.col, pkg.BC_UNDIRECTED | pkg.BC_DIRECTED)
        with pytest.raises(pkg.BCError):  # an asymmetric CSR is not a valid undirected graph
            ctx.load_graph(g.row_ptr, g.col, validate=True)
        bad = g.col.copy()
        bad[0] = g.n  # out of range: refused by the host transpose, with or without BC_VALIDATE
        with pytest.raises(pkg.BCError):
            ctx.load_graph(g.row_ptr, bad, directed=True)
        h = ctx.load_graph(g.row_ptr, g.col, validate=True, directed=True)
        with pytest.raises(pkg.BCError):
            ctx.adaptive_pairs(h, [1, 2], 1.0, 100, 1, 1)
        with pytest.raises(pkg.BCError):
            ctx.submit(h, pkg.BC_QUERY_PAIRS, targets=[1, 2], c=1.0, cap=100, seed=1, qid=1)
        # the context stays usable
        d, _, _ = ctx.source_dependencies(h, [3])
        assert np.array_equal(d[0], oracle.dependencies(g, 3)[0])
        ctx.free_graph(h)
