"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: distances, sigma, draws, stop counts and stop status are bit-exact; the
dependencies, BC and estimates are bit-exact as well because both sides
evaluate every double operation with one rounding and every sum of
dependencies or coefficients as an exact sum rounded once. Where a comparison
is stated with a tolerance, it is the 1e-10 relative bound of the
specification, kept as a guard only.
"""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

WIDTHS = [1, 64]


@pytest.fixture(scope="module")
def pkg():
    import paper_1608_04472_gb300 as p
    return p


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0, batch_width=64)
    yield c
    c.close()


@pytest.fixture(scope="module")
def er2000():
    return gg.erdos_renyi(2000, 8, 1)


def _assert_same(a, b, what):
    a = np.asarray(a)
    b = np.asarray(b)
    if not np.array_equal(a, b):
        diff = np.nonzero(a != b)
        i = tuple(x[0] for x in diff)
        rel = float(np.max(np.abs(a.astype(np.float64) - b) / np.maximum(np.abs(b.astype(np.float64)), 1e-300)))
        raise AssertionError(f"{what}: {len(diff[0])} mismatches, first at {i}: {a[i]} vs {b[i]}, max rel {rel:.3g}")


# ------------------------------------------------------------------ draws --

def test_draw_sources_match_oracle(ctx):
    for n in [1, 2, 7, 2000, 1 << 20, 2_000_000]:
        for i0 in [0, 5, 2**40]:
            got = ctx.draw_sources(123, 9, i0, 300, n)
            exp = [oracle.draw_source(123, 9, i0 + i, n) for i in range(300)]
            _assert_same(got, exp, f"sources n={n} i0={i0}")


def test_draw_pairs_match_oracle(ctx):
    for n in [2, 3, 2000, 2_000_000]:
        s, t = ctx.draw_pairs(77, 2**63 + 5, 17, 200, n)
        exp = [oracle.draw_pair(77, 2**63 + 5, 17 + i, n) for i in range(200)]
        _assert_same(s, [e[0] for e in exp], f"pair s n={n}")
        _assert_same(t, [e[1] for e in exp], f"pair t n={n}")
        assert np.all(s != t)


# -------------------------------------------------------------- exact sum --

def test_exact_sum_matches_fsum(ctx):
    rng = np.random.default_rng(5)
    for trial in range(60):
        k = int(rng.integers(1, 3000))
        lo, hi = sorted(rng.uniform(-76, 40, size=2))
        x = np.exp2(rng.uniform(lo, hi, size=k)) * rng.uniform(1, 2, size=k)
        x = x[(x >= 2.0**-76) & (x < 2.0**62)]
        assert ctx.exact_sum(x) == math.fsum(x)
    assert ctx.exact_sum([1.0, 2.0**-53]) == 1.0
    assert ctx.exact_sum([1.0, 2.0**-53, 2.0**-70]) == 1.0 + 2.0**-52
    assert ctx.exact_sum([0.1] * 10) == 1.0
    assert ctx.exact_sum([]) == 0.0


def test_exact_sum_range_error(ctx, pkg):
    with pytest.raises(pkg.BCError) as e:
        ctx.exact_sum([1.0, 2.0**-90])
    assert e.value.code == -10


# ------------------------------------------------------ per-source step --

def _check_sources(ctx, g, sources, width):
    ctx.set_batch_width(width)
    h = ctx.load_graph(g.row_ptr, g.col, validate=True)
    try:
        delta, dist, sigma = ctx.source_dependencies(h, sources, want_dist=True, want_sigma=True)
    finally:
        ctx.free_graph(h)
        ctx.set_batch_width(64)
    for i, s in enumerate(sources):
        d_o, dist_o, sig_o, ovf = oracle.dependencies(g, int(s))
        assert not ovf
        _assert_same(dist[i], dist_o, f"{g.name} dist s={s} w={width}")
        _assert_same(sigma[i], sig_o, f"{g.name} sigma s={s} w={width}")
        _assert_same(delta[i], d_o, f"{g.name} delta s={s} w={width}")


@pytest.mark.parametrize("width", WIDTHS)
def test_dependencies_er2000(ctx, er2000, width):
    rng = np.random.default_rng(0)
    srcs = rng.integers(0, er2000.n, size=70 if width == 64 else 6).astype(np.int32)  # 64 + ragged 6
    srcs[:2] = [0, er2000.n - 1]
    _check_sources(ctx, er2000, srcs, width)


@pytest.mark.parametrize("width", WIDTHS)
def test_dependencies_rmat_s12_with_hubs(ctx, width):
    # edge factor 64: the top vertices exceed the heavy-degree split (256) many
    # times over, so they are split into several 256-neighbour segments
    g = gg.rmat(12, 64, 0.57, 0.19, 0.19, 3)
    assert g.degrees().max() > 2048
    srcs = np.array([0, 1, 2, 100, 4095, int(np.argmax(g.degrees() == 0))], np.int32)
    _check_sources(ctx, g, srcs, width)


@pytest.mark.parametrize("width", WIDTHS)
def test_dependencies_ba_and_grid(ctx, width):
    _check_sources(ctx, gg.barabasi_albert(3000, 3, 4), np.array([0, 7, 2999], np.int32), width)
    _check_sources(ctx, gg.grid(30), np.array([0, 29, 465, 899], np.int32), width)


def test_duplicate_sources_in_one_batch(ctx, er2000):
    _check_sources(ctx, er2000, np.array([3, 3, 3, 10, 3], np.int32), 64)


def test_tiny_graphs(ctx):
    for edges, n in [([], 1), ([], 3), ([(0, 1)], 2), ([(0, 1), (1, 2)], 3)]:
        e = np.array(edges, np.int32).reshape(-1, 2)
        g = gg.from_edges(n, e[:, 0], e[:, 1])
        for w in WIDTHS:
            _check_sources(ctx, g, np.arange(n, dtype=np.int32), w)


def test_sigma_overflow_boundary(ctx, pkg):
    g = gg.grid(35)  # corner-to-corner sigma C(68,34) > 2^64: the extended form
    h = ctx.load_graph(g.row_ptr, g.col)
    try:
        for w in WIDTHS:
            ctx.set_batch_width(w)
            # from (0,0) the far corner has C(68,34) > 2^64 paths; from (0,1) C(67,33) < 2^64
            d, _, _, _, tier = ctx.source_dependencies_ext(h, [0, 1])
            assert tier.tolist() == [1, 0]
            assert np.array_equal(d[0], oracle.dependencies(g, 0)[0])
            assert np.array_equal(d[1], oracle.dependencies(g, 1)[0])
        g34 = gg.grid(34)
        h2 = ctx.load_graph(g34.row_ptr, g34.col)
        _, _, sig = ctx.source_dependencies(h2, [0], want_sigma=True)
        assert int(sig[0, -1]) == math.comb(66, 33)
        assert ctx.source_dependencies_ext(h2, [0])[4].tolist() == [0]
        ctx.free_graph(h2)
    finally:
        ctx.set_batch_width(64)
        ctx.free_graph(h)


# ------------------------------------------------------------- exact BC --

@pytest.mark.parametrize("width", WIDTHS)
def test_exact_bc_er2000(ctx, er2000, width):
    ctx.set_batch_width(width)
    h = ctx.load_graph(er2000.row_ptr, er2000.col)
    try:
        bc = ctx.exact(h)
    finally:
        ctx.free_graph(h)
        ctx.set_batch_width(64)
    _assert_same(bc, oracle.exact_bc(er2000), f"exact BC w={width}")


def test_exact_bc_closed_forms(ctx):
    n = 37
    path = gg.from_edges(n, np.arange(n - 1), np.arange(1, n))
    star = gg.from_edges(n, np.zeros(n - 1, np.int32), np.arange(1, n))
    h = ctx.load_graph(path.row_ptr, path.col)
    assert ctx.exact(h).tolist() == [2.0 * i * (n - 1 - i) for i in range(n)]
    ctx.free_graph(h)
    h = ctx.load_graph(star.row_ptr, star.col)
    bc = ctx.exact(h)
    assert bc[0] == (n - 1) * (n - 2) and np.all(bc[1:] == 0)
    ctx.free_graph(h)


# --------------------------------------------------------------- uniform --

def test_uniform_estimate_rmat_s12(ctx):
    g = gg.rmat(12, 16, 0.57, 0.19, 0.19, 2)
    k, seed, qid = 150, 4, 8  # two full batches and a ragged tail of 22
    ref = oracle.uniform_sources(g, k, seed, qid)
    h = ctx.load_graph(g.row_ptr, g.col)
    try:
        outs = {}
        for w in WIDTHS:
            ctx.set_batch_width(w)
            outs[w] = ctx.uniform_sources(h, k, seed, qid)
    finally:
        ctx.set_batch_width(64)
        ctx.free_graph(h)
    _assert_same(outs[64], ref, "uniform batched")
    _assert_same(outs[1], ref, "uniform plain")


# ---------------------------------------------------------- Bader (Sec. 4) --

def test_adaptive_sources_small_er_config(ctx, er2000):
    """ER n=2000, average degree 8, seed 1; c=5, 16 uniform targets, cap 64n."""
    targets = gg.uniform_targets(er2000.n, 16, 1)
    c, cap, seed, qid = 5.0, 64 * er2000.n, 1, 1
    ref = oracle.adaptive_sources(er2000, targets, c, cap, seed, qid)
    h = ctx.load_graph(er2000.row_ptr, er2000.col)
    try:
        for w in WIDTHS:
            ctx.set_batch_width(w)
            res = ctx.adaptive_sources(h, targets, c, cap, seed, qid)
            _assert_same(res["k"], ref["k"], f"k w={w}")
            _assert_same(res["status"], ref["status"], f"status w={w}")
            _assert_same(res["S"], ref["S"], f"S w={w}")
            _assert_same(res["est"], ref["est"], f"est w={w}")
    finally:
        ctx.set_batch_width(64)
        ctx.free_graph(h)


def test_adaptive_sources_cap_and_edges(ctx, er2000, pkg):
    h = ctx.load_graph(er2000.row_ptr, er2000.col)
    try:
        res = ctx.adaptive_sources(h, [0, 1, 2], 1e12, 100, 3, 3)  # all capped, ragged last batch
        ref = oracle.adaptive_sources(er2000, [0, 1, 2], 1e12, 100, 3, 3)
        _assert_same(res["k"], ref["k"], "k")
        assert np.all(res["status"] == pkg.BC_CAPPED)
        _assert_same(res["est"], ref["est"], "est")
        for bad in [dict(c=0.5), dict(cap=0)]:
            args = dict(c=2.0, cap=10)
            args.update(bad)
            with pytest.raises(pkg.BCError):
                ctx.adaptive_sources(h, [0], args["c"], args["cap"], 1, 1)
        with pytest.raises(pkg.BCError):
            ctx.adaptive_sources(h, [5, 5], 2.0, 10, 1, 1)
        with pytest.raises(pkg.BCError):
            ctx.adaptive_sources(h, [er2000.n], 2.0, 10, 1, 1)
        empty = ctx.adaptive_sources(h, [], 2.0, 10, 1, 1)
        assert empty["k"].size == 0
    finally:
        ctx.free_graph(h)


# ----------------------------------------------------- pairs (Algorithm 1) --

@pytest.mark.parametrize("scale_kind", ["paper", "n-1"])
def test_adaptive_pairs_ba(ctx, scale_kind):
    g = gg.barabasi_albert(1500, 4, 3)
    targets = gg.degree_targets(g, 5, 3)
    scale = 1.0 if scale_kind == "paper" else float(g.n - 1)
    c, cap, seed, qid = 1.0, 700, 3, 12
    ref = oracle.adaptive_pairs(g, targets, c, cap, seed, qid, threshold_scale=scale)
    h = ctx.load_graph(g.row_ptr, g.col)
    try:
        for w in WIDTHS:
            ctx.set_batch_width(w)
            res = ctx.adaptive_pairs(h, targets, c, cap, seed, qid, threshold_scale=scale)
            _assert_same(res["k"], ref["k"], f"k w={w}")
            _assert_same(res["status"], ref["status"], f"status w={w}")
            _assert_same(res["S"], ref["S"], f"S w={w}")
            _assert_same(res["est"], ref["est"], f"est w={w}")
    finally:
        ctx.set_batch_width(64)
        ctx.free_graph(h)


def test_adaptive_pairs_disconnected(ctx):
    # two components: pairs across them have sigma_st = 0
    e1 = [(i, i + 1) for i in range(9)]
    e2 = [(10 + i, 11 + i) for i in range(5)] + [(10, 15)]
    e = np.array(e1 + e2, np.int32)
    g = gg.from_edges(20, e[:, 0], e[:, 1])  # vertices 16..19 isolated
    targets = np.array([4, 12], np.int32)
    ref = oracle.adaptive_pairs(g, targets, 1.0, 300, 9, 9)
    h = ctx.load_graph(g.row_ptr, g.col)
    try:
        for w in WIDTHS:
            ctx.set_batch_width(w)
            res = ctx.adaptive_pairs(h, targets, 1.0, 300, 9, 9)
            for key in ["k", "status", "S", "est"]:
                _assert_same(res[key], ref[key], f"{key} w={w}")
    finally:
        ctx.set_batch_width(64)
        ctx.free_graph(h)


# ------------------------------------------------------ graph validation --

def test_graph_validation(ctx, pkg):
    rp = np.array([0, 1, 1], np.int32)  # asymmetric
    with pytest.raises(pkg.BCError) as e:
        ctx.load_graph(rp, np.array([1], np.int32), validate=True)
    assert e.value.code == -4
    rp = np.array([0, 1, 2], np.int32)  # self loop
    with pytest.raises(pkg.BCError):
        ctx.load_graph(rp, np.array([0, 1], np.int32), validate=True)
    rp = np.array([0, 2, 3, 4], np.int32)  # unsorted row
    with pytest.raises(pkg.BCError):
        ctx.load_graph(rp, np.array([2, 1, 0, 0], np.int32), validate=True)
    with pytest.raises(pkg.BCError) as e:
        ctx.exact(12345)
    assert e.value.code == -8


# ------------------------------------------------- full-size sampled parity --

@pytest.fixture(scope="module")
def rmat20():
    return gg.rmat(20, 16, 0.57, 0.19, 0.19, 2)


def test_rmat20_sampled_sources(ctx, rmat20):
    """R-MAT scale 20 at full size: per-source dist/sigma/delta for a few sources,
    in the 64-wide launch configuration the benchmark uses."""
    srcs = ctx.draw_sources(2, 1, 0, 64, rmat20.n)  # one full batch
    h = ctx.load_graph(rmat20.row_ptr, rmat20.col)
    try:
        delta, dist, sigma = ctx.source_dependencies(h, srcs, want_dist=True, want_sigma=True)
    finally:
        ctx.free_graph(h)
    for i in [0, 1, 17, 63]:
        d_o, dist_o, sig_o, _ = oracle.dependencies(rmat20, int(srcs[i]))
        _assert_same(dist[i], dist_o, f"dist lane {i}")
        _assert_same(sigma[i], sig_o, f"sigma lane {i}")
        _assert_same(delta[i], d_o, f"delta lane {i}")


def test_rmat20_bader_first_draws(ctx, rmat20):
    """Bader's loop on R-MAT s20 with 512 uniform targets, c=5, capped at 66 draws
    (a full batch plus a ragged one): k, S and est bit-exact."""
    targets = gg.uniform_targets(rmat20.n, 512, 2)
    h = ctx.load_graph(rmat20.row_ptr, rmat20.col)
    try:
        res = ctx.adaptive_sources(h, targets, 5.0, 66, 2, 1)
    finally:
        ctx.free_graph(h)
    ref = oracle.adaptive_sources(rmat20, targets, 5.0, 66, 2, 1)
    for key in ["k", "status", "S", "est"]:
        _assert_same(res[key], ref[key], key)


# ------------------------------------------- pairs at the BA workload's size --

@pytest.fixture(scope="module")
def ba2m():
    """Barabasi-Albert n=2,000,000, 4 edges per new vertex, seed 3."""
    return gg.barabasi_albert(2_000_000, 4, 3)


def test_ba2m_pairs_sampled(ctx, ba2m):
    """Algorithm 1 on the full-size BA graph with degree-proportional targets and
    the 64-wide pair batches: 4 targets and the top hub, cap 70 draws (a full batch + a ragged
    one), literal threshold c*n; k, S, status and est bit-exact."""
    targets = np.concatenate([gg.degree_targets(ba2m, 4, 3),
                              [int(np.argmax(ba2m.degrees()))]]).astype(np.int32)  # + the top hub
    targets = np.unique(targets)
    h = ctx.load_graph(ba2m.row_ptr, ba2m.col)
    try:
        res = ctx.adaptive_pairs(h, targets, 1.0, 70, 3, 21)
    finally:
        ctx.free_graph(h)
    ref = oracle.adaptive_pairs(ba2m, targets, 1.0, 70, 3, 21)
    for key in ["k", "status", "S", "est"]:
        _assert_same(res[key], ref[key], key)


def test_ba20k_pairs_full_run():
    """A complete Algorithm 1 run (every target stops before its cap under the
    Bader-scaled test S*(n-1) > c*n) on BA n=20,000 built like the 2M workload."""
    import paper_1608_04472_gb300 as pkg
    g = gg.barabasi_albert(20_000, 4, 3)
    targets = np.argsort(-g.degrees(), kind="stable")[:8].astype(np.int32)  # the hubs: high BC
    scale = float(g.n - 1)
    ref = oracle.adaptive_pairs(g, targets, 2.0, 6000, 4, 4, threshold_scale=scale)
    with pkg.Context(0, batch_width=64) as c:
        h = c.load_graph(g.row_ptr, g.col)
        res = c.adaptive_pairs(h, targets, 2.0, 6000, 4, 4, threshold_scale=scale)
    for key in ["k", "status", "S", "est"]:
        _assert_same(res[key], ref[key], key)
    assert np.all(res["status"] == pkg.BC_STOPPED)


@pytest.mark.parametrize("shape", ["edgeless", "matching", "star", "two_stars"])
def test_source_key_degenerate_graphs(ctx, shape):
    """Graphs where the source key's landmarks run out early (every vertex
    reached from the hub is a landmark), its distances have no spread (zero
    covariance) or most vertices are not reached from the hub (key 255): the
    uniform estimate, exact BC and Bader's loop equal the oracle's."""
    n = 60
    if shape == "edgeless":
        u, v = np.zeros(0, np.int32), np.zeros(0, np.int32)
    elif shape == "matching":
        u, v = np.arange(0, 40, 2, dtype=np.int32), np.arange(1, 40, 2, dtype=np.int32)
    elif shape == "star":
        u, v = np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32)
    else:
        u = np.concatenate([np.zeros(29, np.int32), np.full(29, 30, np.int32)])
        v = np.concatenate([np.arange(1, 30, dtype=np.int32), np.arange(31, 60, dtype=np.int32)])
    g = gg.from_edges(n, u, v)
    h = ctx.load_graph(g.row_ptr, g.col)
    try:
        _assert_same(ctx.uniform_sources(h, 300, 4, 6), oracle.uniform_sources(g, 300, 4, 6), "uniform")
        _assert_same(ctx.exact(h), oracle.exact_bc(g), "exact")
        targets = [0, 1, 30, 59]
        res = ctx.adaptive_sources(h, targets, 1.5, 400, 4, 7)
        ref = oracle.adaptive_sources(g, targets, 1.5, 400, 4, 7)
        for key in ("k", "S", "status", "est"):
            _assert_same(res[key], ref[key], key)
    finally:
        ctx.free_graph(h)
