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


@pytest.mark.parametrize("width", [1, 64])
def test_pairs_on_overflowing_grid(pkg, width):
    # corner targets and far pairs (distance > ~70 on a 60x60 grid) have counts
    # beyond 2^64: targets and pair lanes are recomputed in the extended form
    g = gg.grid(60)
    targets = [0, g.n - 1, 30 * 60 + 30, 61, 5 * 60 + 53]
    far = sum(1 for s, t in (oracle.draw_pair(1, 1, i, g.n) for i in range(60))
              if abs(s // 60 - t // 60) + abs(s % 60 - t % 60) > 75)
    assert far >= 1  # the draws include pairs whose sigma_st overflows
    cap = 200 if width == 64 else 60
    ref = oracle.adaptive_pairs(g, targets, 1.0, cap, 1, 1)
    ref2 = oracle.adaptive_pairs(g, targets, 2.0, 3 * cap, 2, 5, float(g.n - 1))
    with pkg.Context(0, batch_width=width) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        got = ctx.adaptive_pairs(h, targets, 1.0, cap, 1, 1)
        got2 = ctx.adaptive_pairs(h, targets, 2.0, 3 * cap, 2, 5, float(g.n - 1))
        tk = ctx.submit(h, pkg.BC_QUERY_PAIRS, targets=targets, c=1.0, cap=cap, seed=1, qid=1)
        assert ctx.poll(tk, -1) == pkg.BC_OK
        served = tk.outputs()
    for key in ["est", "k", "S", "status"]:
        assert np.array_equal(got[key], ref[key]), key
        assert np.array_equal(got2[key], ref2[key]), key
        assert np.array_equal(served[key], ref[key]), key
    assert np.sum(ref["S"] > 0) >= 2
