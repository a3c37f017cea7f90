"""GPU parity of the extended form: samples whose path counts exceed 2^64-1
(grids from a corner: sigma = C(i+j, i)) are recomputed with doubles of
unbounded exponent. Every result must equal the oracle bit for bit, for both
the plain (width 1) and the 64-lane batched engine, with batches that mix
lanes of both forms."""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1608_04472_gb300 as p
    return p


def _xf_from_u64(sig):
    """(mantissa in [1,2), exponent) of RN(sigma) for uint64 counts."""
    m = np.zeros(sig.shape, np.float64)
    e = np.zeros(sig.shape, np.int64)
    for i, x in enumerate(sig.ravel().tolist()):
        if x:
            f, k = math.frexp(float(x))
            m.ravel()[i], e.ravel()[i] = 2.0 * f, k - 1
    return m, e


def _expected(g, sources):
    rows = []
    for s in sources:
        delta, dist, sig, ovf = oracle.dependencies(g, s)
        if ovf:
            _, _, sm, se = oracle.dependencies_xf(g, s)
        else:
            sm, se = _xf_from_u64(sig)
        rows.append((delta, dist, sm, se, int(ovf)))
    return rows


@pytest.mark.parametrize("width", [1, 64])
@pytest.mark.parametrize("side", [40, 150])
def test_grid_sources_match_oracle(pkg, width, side):
    g = gg.grid(side)
    c = side // 2
    # corners and edges overflow; sources near the centre of the 40-grid do not
    sources = [0, side - 1, g.n - 1, c * side + c, c * side, 3 * side + 7, c * side + c, 1]
    exp = _expected(g, sources)
    assert any(r[4] for r in exp)
    if side == 40:
        assert not all(r[4] for r in exp)
    with pkg.Context(0, batch_width=width) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        delta, dist, sm, se, tier = ctx.source_dependencies_ext(h, sources)
        d2, dist2, sig2 = ctx.source_dependencies(h, sources, want_dist=True, want_sigma=True)
    for i, (ed, edist, esm, ese, eovf) in enumerate(exp):
        assert tier[i] == eovf, i
        assert np.array_equal(dist[i], edist), i
        assert np.array_equal(delta[i], ed), (i, np.sum(delta[i] != ed))
        assert np.array_equal(sm[i], esm), i
        assert np.array_equal(se[i].astype(np.int64), ese), i
        assert np.array_equal(d2[i], ed) and np.array_equal(dist2[i], edist)
        if eovf:
            assert np.all(sig2[i][edist >= 0] == np.uint64(2**64 - 1)) and np.all(sig2[i][edist < 0] == 0)
        else:
            assert np.array_equal(sig2[i], oracle.bfs(g, sources[i])[1])


@pytest.mark.parametrize("width", [1, 64])
def test_exact_bc_on_grid_with_mixed_forms(pkg, width):
    g = gg.grid(36)  # corner sources overflow, central ones do not
    ref = oracle.exact_bc(g)
    with pkg.Context(0, batch_width=width) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        got = ctx.exact(h)
    assert np.array_equal(got, ref), np.sum(got != ref)


def test_uniform_and_bader_on_grid(pkg):
    g = gg.grid(48)
    ref_u = oracle.uniform_sources(g, 200, 7, 3)
    targets = gg.uniform_targets(g.n, 12, 5)
    ref_b = oracle.adaptive_sources(g, targets, 2.0, 700, 9, 4)
    with pkg.Context(0, batch_width=64) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        got_u = ctx.uniform_sources(h, 200, 7, 3)
        got_b = ctx.adaptive_sources(h, targets, 2.0, 700, 9, 4)
        tk = ctx.submit(h, pkg.BC_QUERY_SOURCES, targets=targets, c=2.0, cap=700, seed=9, qid=4)
        assert ctx.poll(tk, -1) == pkg.BC_OK
        served = tk.outputs()
    assert np.array_equal(got_u, ref_u), np.sum(got_u != ref_u)
    for key in ["est", "k", "S", "status"]:
        assert np.array_equal(got_b[key], ref_b[key]), key
        assert np.array_equal(served[key], ref_b[key]), key


def test_pairs_on_overflowing_grid_report_overflow(pkg):
    g = gg.grid(40)
    with pkg.Context(0, batch_width=64) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        with pytest.raises(pkg.BCError) as e:
            ctx.adaptive_pairs(h, [0, g.n - 1], 1.0, 64, 1, 1)
        assert e.value.code == -9
        # the context stays usable
        d, _, _ = ctx.source_dependencies(h, [5])
        assert np.array_equal(d[0], oracle.dependencies(g, 5)[0])
