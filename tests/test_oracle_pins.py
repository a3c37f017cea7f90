"""Pins for the CPU oracle: checks against what the paper and mathematics fix.

Nothing here compares the oracle with itself. The pins are:
  * Philox4x64-10 against numpy's independent Philox bit generator;
  * the exact sum against Python's math.fsum (correctly rounded summation);
  * shortest-path counts against binomial closed forms on grids (exact ints);
  * BC against closed forms (path, star, cycles, complete and complete
    bipartite graphs), against brute-force enumeration of every shortest path
    on small graphs (exact rationals), and against networkx (x2: ordered pairs);
  * the invariant sum_v delta_s(v) = sum_t (d(s,t) - 1) (each s-t shortest path
    has d(s,t)-1 interior vertices);
  * the pair formula of Algorithm 1 against Def. 1 (sum over all pairs = BC);
  * stop rules against a plain re-run of the loop on the logged draws;
  * unbiasedness E[X_i] = A/n (Corollary 1) and E[Y_i] = A/(n(n-1)) (Corollary 3).
"""
import itertools
import math
from fractions import Fraction

import networkx as nx
import numpy as np
import pytest

import graphgen as gg
import oracle

# ------------------------------------------------------------------ helpers --


def graph_from_edges(n, edges, name="g"):
    e = np.array(edges, dtype=np.int32).reshape(-1, 2)
    return gg.from_edges(n, e[:, 0], e[:, 1], name)


def nx_graph(g):
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(g.edges().tolist())
    return G


def brute_paths(g):
    """All shortest paths between every ordered pair, by enumerating every simple
    path (no BFS): returns dict (s,t) -> list of vertex tuples."""
    adj = [set(g.neighbors(v).tolist()) for v in range(g.n)]
    out = {}
    for s in range(g.n):
        paths = {}

        def dfs(path, seen):
            v = path[-1]
            paths.setdefault(v, []).append(tuple(path))
            for w in adj[v]:
                if w not in seen:
                    seen.add(w)
                    path.append(w)
                    dfs(path, seen)
                    path.pop()
                    seen.discard(w)

        dfs([s], {s})
        for t, ps in paths.items():
            if t == s:
                continue
            L = min(len(p) for p in ps)
            out[(s, t)] = [p for p in ps if len(p) == L]
    return out


def brute_bc_and_delta(g):
    """Exact rational BC(v) (Def. 1, ordered pairs) and delta_s(v) (Def. 2)."""
    sp = brute_paths(g)
    bc = [Fraction(0)] * g.n
    delta = [[Fraction(0)] * g.n for _ in range(g.n)]
    for (s, t), ps in sp.items():
        sig = len(ps)
        for v in range(g.n):
            if v in (s, t):
                continue
            through = sum(1 for p in ps if v in p)
            if through:
                f = Fraction(through, sig)
                bc[v] += f
                delta[s][v] += f
    return bc, delta


def rel_close(a, b, tol):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.all(np.abs(a - b) <= tol * np.maximum(np.abs(b), 1.0))


# ------------------------------------------------------------------- Philox --


def _numpy_philox_block(counter, key):
    c = (counter - 1) % (1 << 256)  # numpy increments the counter before use
    ctr = np.array([(c >> (64 * j)) & (2**64 - 1) for j in range(4)], dtype=np.uint64)
    bg = np.random.Philox(counter=ctr, key=np.array(key, dtype=np.uint64))
    return [int(x) for x in bg.random_raw(4)]


@pytest.mark.parametrize("counter,key", [
    (0, (0, 0)), (1, (0, 0)), (0, (1, 2)), (12345, (2**64 - 1, 7)),
    ((5 << 64) | 3, (99, 2**63)), ((1 << 255) | 17, (0xDEADBEEF, 0xCAFEF00D)),
])
def test_philox_matches_numpy(counter, key):
    words = [(counter >> (64 * j)) & (2**64 - 1) for j in range(4)]
    assert oracle.philox4x64_10(words, list(key)) == _numpy_philox_block(counter, key)


def test_draw_source_matches_numpy_mapping():
    seed, qid, n = 77, 5, 1_000_003
    for i in [0, 1, 2, 1000, 2**33]:
        x0 = _numpy_philox_block(i, (seed, qid))[0]
        assert oracle.draw_source(seed, qid, i, n) == (x0 * n) >> 64


def test_draw_source_uniform():
    n, N = 7, 70000
    counts = np.bincount([oracle.draw_source(3, 4, i, n) for i in range(N)], minlength=n)
    chi2 = float(np.sum((counts - N / n) ** 2 / (N / n)))
    assert chi2 < 30.0  # chi-square, 6 dof; p ~ 4e-5


def test_draw_pair_uniform_ordered_distinct():
    n, N = 5, 60000
    counts = {}
    for i in range(N):
        u, t = oracle.draw_pair(11, 12, i, n)
        assert 0 <= u < n and 0 <= t < n and u != t
        counts[(u, t)] = counts.get((u, t), 0) + 1
    assert len(counts) == n * (n - 1)
    exp = N / (n * (n - 1))
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 60.0  # 19 dof


# ---------------------------------------------------------------- exact sum --


def test_exact_sum_matches_fsum_random():
    rng = np.random.default_rng(0)
    for _ in range(3000):
        k = int(rng.integers(1, 64))
        lo, hi = sorted(rng.uniform(-1080, 1000, size=2))
        x = np.exp2(rng.uniform(lo, hi, size=k)) * rng.uniform(1, 2, size=k)
        x = x[np.isfinite(x)]
        assert oracle.exact_sum(x) == math.fsum(x)


def test_exact_sum_special_cases():
    tiny = np.nextafter(0.0, 1.0)
    cases = [
        [1.0, 2.0**-53],                # tie -> even (1.0)
        [1.0, 2.0**-53, 2.0**-80],      # just above the tie -> up
        [1.0 + 2.0**-52, 2.0**-53],     # tie -> even (up)
        [tiny] * 5,                     # subnormals
        [0.1] * 10,
        [2.0**1000, 2.0**-1000],
        [0.0, 0.0],
        [1e308, 1e307],
    ]
    for c in cases:
        assert oracle.exact_sum(c) == math.fsum(c), c
    assert oracle.exact_sum([1.0, 2.0**-53]) == 1.0
    assert oracle.exact_sum([0.1] * 10) == 1.0


def test_exact_sum_order_independent():
    rng = np.random.default_rng(1)
    x = np.exp2(rng.uniform(-100, 30, size=500))
    a = oracle.exact_sum(x)
    for _ in range(5):
        assert oracle.exact_sum(rng.permutation(x)) == a


# ------------------------------------------------------------- sigma / dist --


@pytest.mark.parametrize("side", [1, 2, 7, 12])
def test_grid_sigma_is_binomial(side):
    g = gg.grid(side)
    dist, sigma, order, ovf = oracle.bfs(g, 0)
    assert not ovf
    for i in range(side):
        for j in range(side):
            v = i * side + j
            assert dist[v] == i + j
            assert int(sigma[v]) == math.comb(i + j, i)
    # order lists vertices by non-decreasing distance
    assert np.all(np.diff(dist[order]) >= 0)


def test_sigma_overflow_flag():
    # corner-to-corner sigma = C(2(side-1), side-1): C(66,33) < 2^64 < C(68,34)
    assert math.comb(66, 33) < 2**64 < math.comb(68, 34)
    _, sigma, _, ovf = oracle.bfs(gg.grid(34), 0)
    assert not ovf and int(sigma[-1]) == math.comb(66, 33)
    _, _, _, ovf = oracle.bfs(gg.grid(35), 0)
    assert ovf


def test_unreachable_and_isolated():
    g = graph_from_edges(6, [(0, 1), (1, 2), (4, 5)])
    dist, sigma, order, _ = oracle.bfs(g, 0)
    assert dist.tolist() == [0, 1, 2, -1, -1, -1]
    assert sigma.tolist() == [1, 1, 1, 0, 0, 0]
    delta, _, _, _ = oracle.dependencies(g, 3)  # isolated source
    assert np.all(delta == 0)
    delta, _, _, _ = oracle.dependencies(g, 0)
    assert delta.tolist() == [0.0, 1.0, 0.0, 0.0, 0.0, 0.0]


# ------------------------------------------------------------- closed forms --


def test_path_closed_form():
    for n in [2, 3, 5, 17]:
        g = graph_from_edges(n, [(i, i + 1) for i in range(n - 1)])
        bc = oracle.exact_bc(g)
        assert bc.tolist() == [2.0 * i * (n - 1 - i) for i in range(n)]


def test_star_closed_form():
    for n in [3, 4, 10, 50]:
        g = graph_from_edges(n, [(0, i) for i in range(1, n)])
        bc = oracle.exact_bc(g)
        assert bc[0] == (n - 1) * (n - 2)
        assert np.all(bc[1:] == 0)


def test_cycle_closed_form():
    for k in [2, 3, 6]:
        n = 2 * k + 1
        g = graph_from_edges(n, [(i, (i + 1) % n) for i in range(n)])
        assert np.allclose(oracle.exact_bc(g), k * (k - 1), rtol=1e-14)
    for k in [2, 3, 7]:
        n = 2 * k
        g = graph_from_edges(n, [(i, (i + 1) % n) for i in range(n)])
        assert np.allclose(oracle.exact_bc(g), (k - 1) ** 2, rtol=1e-14)


def test_complete_and_bipartite_closed_forms():
    for n in [2, 3, 8]:
        g = graph_from_edges(n, list(itertools.combinations(range(n), 2)))
        assert np.all(oracle.exact_bc(g) == 0)
    for a, b in [(2, 3), (3, 5), (4, 4)]:
        g = graph_from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)])
        bc = oracle.exact_bc(g)
        assert np.allclose(bc[:a], b * (b - 1) / a, rtol=1e-14)
        assert np.allclose(bc[a:], a * (a - 1) / b, rtol=1e-14)


# -------------------------------------------------------------- brute force --


def _random_small(n, p, seed):
    rng = np.random.default_rng(seed)
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    return graph_from_edges(n, edges)


@pytest.mark.parametrize("seed", range(24))
def test_bruteforce_random_small(seed):
    n = 3 + seed % 7
    g = _random_small(n, 0.25 + 0.05 * (seed % 8), seed)
    bc_b, delta_b = brute_bc_and_delta(g)
    bc = oracle.exact_bc(g)
    assert rel_close(bc, [float(x) for x in bc_b], 1e-13)
    for s in range(n):
        delta, _, _, _ = oracle.dependencies(g, s)
        assert rel_close(delta, [float(x) for x in delta_b[s]], 1e-13)


def test_bruteforce_all_graphs_on_5_vertices():
    pairs = list(itertools.combinations(range(5), 2))
    for mask in range(1 << len(pairs)):
        edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        g = graph_from_edges(5, edges)
        bc_b, _ = brute_bc_and_delta(g)
        assert rel_close(oracle.exact_bc(g), [float(x) for x in bc_b], 1e-14), edges


# --------------------------------------------------------------- invariants --


@pytest.mark.parametrize("family", ["er", "rmat", "ba"])
def test_dependency_sum_invariant(family):
    g = {"er": lambda: gg.erdos_renyi(400, 6, 9),
         "rmat": lambda: gg.rmat(10, 8, 0.57, 0.19, 0.19, 4),
         "ba": lambda: gg.barabasi_albert(600, 3, 2)}[family]()
    for s in [0, 1, g.n // 2, g.n - 1]:
        delta, dist, _, _ = oracle.dependencies(g, s)
        reach = dist > 0
        expect = float(np.sum(dist[reach] - 1))
        assert math.isclose(math.fsum(delta), expect, rel_tol=1e-12, abs_tol=1e-9)


def test_bc_total_invariant():
    g = gg.erdos_renyi(300, 4, 3)
    bc = oracle.exact_bc(g)
    total = 0
    for s in range(g.n):
        dist, _, _, _ = oracle.bfs(g, s)
        total += int(np.sum(dist[dist > 0] - 1))
    assert math.isclose(math.fsum(bc), total, rel_tol=1e-12)


def test_networkx_er2000():
    """The small ER workload: n=2000, average degree 8, seed 1."""
    g = gg.erdos_renyi(2000, 8, 1)
    bc = oracle.exact_bc(g)
    ref = nx.betweenness_centrality(nx_graph(g), normalized=False)
    ref = 2.0 * np.array([ref[i] for i in range(g.n)])
    assert rel_close(bc, ref, 1e-10)


def test_networkx_rmat_s10():
    g = gg.rmat(10, 16, 0.57, 0.19, 0.19, 2)
    bc = oracle.exact_bc(g)
    ref = nx.betweenness_centrality(nx_graph(g), normalized=False)
    assert rel_close(bc, 2.0 * np.array([ref[i] for i in range(g.n)]), 1e-10)


def test_exact_bc_is_correctly_rounded_sum_of_dependencies():
    g = gg.rmat(8, 8, 0.57, 0.19, 0.19, 1)
    D = np.stack([oracle.dependencies(g, s)[0] for s in range(g.n)])
    bc = oracle.exact_bc(g)
    for v in range(g.n):
        assert bc[v] == math.fsum(D[:, v])


# --------------------------------------------------------------------- pairs --


def _pair_table(g, v):
    """y(s,t) = sigma_st(v)/sigma_st for every ordered pair via the oracle."""
    dv, sv, _, _ = oracle.bfs(g, v)
    Y = np.zeros((g.n, g.n))
    for s in range(g.n):
        ds, ss, _, _ = oracle.bfs(g, s)
        for t in range(g.n):
            if s != t:
                Y[s, t] = oracle.pair_value(v, s, t, dv, sv, int(ds[t]), int(ss[t]))
    return Y


def test_pair_values_sum_to_bc_bruteforce():
    """Def. 1: summing the pair dependency over all ordered pairs gives BC(v)."""
    for seed in range(6):
        g = _random_small(8, 0.35, 100 + seed)
        bc_b, _ = brute_bc_and_delta(g)
        for v in range(g.n):
            assert math.isclose(math.fsum(_pair_table(g, v).ravel()), float(bc_b[v]),
                                rel_tol=1e-13, abs_tol=1e-12)


def test_pair_values_row_sums_are_dependencies():
    """sum_t sigma_st(v)/sigma_st = delta_s(v): ties Algorithm 1 to Theorem 1."""
    g = gg.barabasi_albert(120, 2, 7)
    for v in [0, 3, 50]:
        Y = _pair_table(g, v)
        for s in range(0, g.n, 7):
            delta, _, _, _ = oracle.dependencies(g, s)
            assert math.isclose(math.fsum(Y[s]), delta[v], rel_tol=1e-12, abs_tol=1e-12)


def test_pair_sequence_matches_draws():
    g = gg.erdos_renyi(200, 5, 2)
    y, s, t = oracle.pair_sequence(g, 17, 5, 6, 10, 50)
    for q in range(50):
        assert (int(s[q]), int(t[q])) == oracle.draw_pair(5, 6, 10 + q, g.n)
    assert np.all(y >= 0) and np.all(y <= 1)


# --------------------------------------------------------------- stop rules --


def test_bader_stop_rule_replayed():
    g = gg.erdos_renyi(300, 6, 5)
    targets = [0, 7, 150, 299]
    c, cap, seed, qid = 1.5, 400, 21, 3
    res = oracle.adaptive_sources(g, targets, c, cap, seed, qid)
    n = g.n
    for j, v in enumerate(targets):
        S, k, stopped = 0.0, 0, False
        for i in range(cap):
            s = oracle.draw_source(seed, qid, i, n)
            S = S + oracle.dependencies(g, s)[0][v]
            k = i + 1
            if S > c * n:
                stopped = True
                break
        assert res["k"][j] == k and res["S"][j] == S
        assert res["status"][j] == (oracle.STOPPED if stopped else oracle.CAPPED)
        assert res["est"][j] == (n * S) / k


def test_pairs_stop_rule_replayed():
    g = gg.erdos_renyi(60, 4, 8)
    targets = [3, 30]
    c, cap, seed, qid = 1.0, 3000, 4, 9
    for scale in [1.0, float(g.n - 1)]:
        res = oracle.adaptive_pairs(g, targets, c, cap, seed, qid, threshold_scale=scale)
        for j, v in enumerate(targets):
            y, _, _ = oracle.pair_sequence(g, v, seed, qid, 0, int(res["k"][j]))
            S = 0.0
            for i, yi in enumerate(y):
                S = S + yi
                if S * scale > c * g.n:
                    assert i + 1 == res["k"][j] and res["status"][j] == oracle.STOPPED
                    break
            else:
                assert res["k"][j] == cap and res["status"][j] == oracle.CAPPED
            assert res["S"][j] == S
            assert res["est"][j] == (g.n * (g.n - 1.0) * S) / res["k"][j]


def test_cap_and_parameter_validation():
    g = gg.erdos_renyi(50, 3, 1)
    res = oracle.adaptive_sources(g, [0, 1], 1e9, 7, 1, 1)
    assert np.all(res["k"] == 7) and np.all(res["status"] == oracle.CAPPED)
    with pytest.raises(ValueError):
        oracle.adaptive_sources(g, [0], 0.5, 10, 1, 1)  # c >= 1 (Sec. 4 footnote)
    with pytest.raises(ValueError):
        oracle.adaptive_sources(g, [50], 2.0, 10, 1, 1)
    with pytest.raises(ValueError):
        oracle.adaptive_pairs(g, [0], 2.0, 0, 1, 1)


# ------------------------------------------------------------- unbiasedness --


def test_uniform_estimate_is_correctly_rounded():
    g = gg.erdos_renyi(150, 4, 6)
    k, seed, qid = 40, 3, 4
    est = oracle.uniform_sources(g, k, seed, qid)
    D = np.stack([oracle.dependencies(g, oracle.draw_source(seed, qid, i, g.n))[0]
                  for i in range(k)])
    for v in range(g.n):
        assert est[v] == (g.n * math.fsum(D[:, v])) / k


def test_source_sampling_unbiased():
    """Corollary 1: E[X_i] = A/n, so E[n * X_i] = BC(v)."""
    g = gg.erdos_renyi(40, 3, 12)
    bc = oracle.exact_bc(g)
    n = g.n
    D = np.stack([oracle.dependencies(g, s)[0] for s in range(n)])
    # exact expectation over the uniform source distribution
    assert rel_close(n * D.mean(axis=0), bc, 1e-12)
    # empirical: 4000 draws of the Philox stream
    xs = np.array([D[oracle.draw_source(8, 1, i, n)] for i in range(4000)])
    mean, se = n * xs.mean(axis=0), n * xs.std(axis=0) / math.sqrt(len(xs))
    ok = (np.abs(mean - bc) <= 5 * se + 1e-9)
    assert ok.all()


def test_pair_sampling_unbiased():
    """Corollary 3: E[Y_i] = A/(n(n-1)) under uniform ordered distinct pairs."""
    g = _random_small(9, 0.3, 5)
    bc_b, _ = brute_bc_and_delta(g)
    v = int(np.argmax([float(x) for x in bc_b]))
    Y = _pair_table(g, v)
    n = g.n
    ys = np.array([Y[oracle.draw_pair(2, 2, i, n)] for i in range(20000)])
    mean = n * (n - 1) * ys.mean()
    se = n * (n - 1) * ys.std() / math.sqrt(len(ys))
    assert abs(mean - float(bc_b[v])) <= 5 * se
