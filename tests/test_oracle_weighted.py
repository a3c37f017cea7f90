"""Pins for the oracle on weighted graphs (Sec. 3 step 1: Dijkstra; Def. 3
with edge lengths; Theorem 1): unit lengths reproduce the unweighted oracle
bit for bit (including samples in the extended form), networkx's weighted
betweenness, subdividing every edge of length k into k unit edges keeps the
distances and path counts between original vertices, brute-force enumeration
of every shortest path on small graphs with many ties, invariance under
scaling all lengths, binomial counts on a grid of equal lengths beyond 2^64,
and closed forms on a triangle and a square with unequal sides."""
import math
import random
from fractions import Fraction

import networkx as nx
import numpy as np
import pytest

import graphgen as gg
import oracle
from test_oracle_pins import rel_close

U = 2.0**-53


def _ones(g):
    return np.ones(g.col.shape[0], np.uint32)


@pytest.mark.parametrize("make", [
    lambda: gg.erdos_renyi(300, 4, 51),
    lambda: gg.rmat(9, 8, 0.57, 0.19, 0.19, 52),
    lambda: gg.grid(40),  # corner sources beyond 2^64: the extended form
    lambda: gg.directed_rmat(9, 8, 0.57, 0.19, 0.19, 53),
])
def test_unit_lengths_equal_the_unweighted_oracle(make):
    g = make()
    for s in [0, 1, g.n // 2, g.n - 1, 37]:
        d, dist, sig, ovf = oracle.dependencies(g, s)
        dw, distw, sigw, ovfw, smw, sew = oracle.dependencies_w(g, _ones(g), s)
        assert ovf == ovfw, s
        assert np.array_equal(distw, dist.astype(np.int64)), s
        assert np.array_equal(dw, d), (s, np.sum(dw != d))
        if ovf:
            _, _, sm, se = oracle.dependencies_xf(g, s)
            assert np.array_equal(smw, sm) and np.array_equal(sew, se), s
            assert np.all(sigw[dist >= 0] == np.uint64(2**64 - 1)) and np.all(sigw[dist < 0] == 0)
        else:
            assert np.array_equal(sigw, sig), s


def test_unit_length_estimators_equal_the_unweighted_ones():
    g = gg.erdos_renyi(400, 5, 54)
    w = _ones(g)
    assert np.array_equal(oracle.exact_bc_w(g, w), oracle.exact_bc(g))
    assert np.array_equal(oracle.uniform_sources_w(g, w, 50, 3, 4), oracle.uniform_sources(g, 50, 3, 4))
    t = gg.uniform_targets(g.n, 6, 5)
    a = oracle.adaptive_sources_w(g, w, t, 2.0, 300, 6, 7)
    b = oracle.adaptive_sources(g, t, 2.0, 300, 6, 7)
    for key in ["est", "k", "S", "status"]:
        assert np.array_equal(a[key], b[key]), key


def _nx_graph(g, w, directed):
    G = nx.DiGraph() if directed else nx.Graph()
    G.add_nodes_from(range(g.n))
    for u in range(g.n):
        for j in range(g.row_ptr[u], g.row_ptr[u + 1]):
            G.add_edge(u, int(g.col[j]), weight=int(w[j]))
    return G


@pytest.mark.parametrize("directed", [False, True])
def test_weighted_bc_matches_networkx(directed):
    if directed:
        g = gg.directed_er(250, 4, 55)
        w = gg.edge_lengths(g, 1, 6, 56, symmetric=False)
    else:
        g = gg.erdos_renyi(250, 5, 57)
        w = gg.edge_lengths(g, 1, 6, 58)
    ref = nx.betweenness_centrality(_nx_graph(g, w, directed), weight="weight", normalized=False)
    factor = 1.0 if directed else 2.0  # networkx halves undirected BC (ordered pairs here, R1)
    bc = oracle.exact_bc_w(g, w)
    assert rel_close(bc, [factor * ref[v] for v in range(g.n)], 1e-9)


def test_subdividing_edges_keeps_distances_and_counts():
    # an edge {u, v} of length k becomes a path of k unit edges through k-1 new
    # vertices: distances and shortest-path counts between original vertices
    # stay the same
    g = gg.erdos_renyi(120, 4, 59)
    w = gg.edge_lengths(g, 1, 4, 60)
    eu, ev, nxt = [], [], g.n
    for u in range(g.n):
        for j in range(g.row_ptr[u], g.row_ptr[u + 1]):
            v, k = int(g.col[j]), int(w[j])
            if v < u:
                continue
            chain = [u] + list(range(nxt, nxt + k - 1)) + [v]
            nxt += k - 1
            eu += chain[:-1]
            ev += chain[1:]
    h = gg.from_edges(nxt, np.array(eu, np.int32), np.array(ev, np.int32))
    for s in [0, 5, 60, 119]:
        _, dist, sig, _ = oracle.dependencies(h, s)
        _, distw, sigw, ovf, _, _ = oracle.dependencies_w(g, w, s)
        assert not ovf
        assert np.array_equal(distw, dist[: g.n].astype(np.int64)), s
        assert np.array_equal(sigw, sig[: g.n]), s


def _brute_delta_w(n, adj, s):
    """delta_s(v) from every simple path out of s, shortest by total length."""
    best = {}

    def dfs(v, length, path, seen):
        best.setdefault(v, []).append((length, tuple(path)))
        for x, k in adj[v]:
            if x not in seen:
                seen.add(x)
                path.append(x)
                dfs(x, length + k, path, seen)
                path.pop()
                seen.discard(x)

    dfs(s, 0, [s], {s})
    delta = [Fraction(0)] * n
    for t, ps in best.items():
        if t == s:
            continue
        L = min(p[0] for p in ps)
        sp = [p[1] for p in ps if p[0] == L]
        for v in range(n):
            if v not in (s, t):
                c = sum(1 for p in sp if v in p)
                if c:
                    delta[v] += Fraction(c, len(sp))
    return delta


@pytest.mark.parametrize("seed", range(12))
def test_weighted_bruteforce_small(seed):
    rng = random.Random(300 + seed)
    n = 5 + seed % 4
    directed = seed % 3 == 2
    eu, ev = [], []
    for u in range(n):
        for v in range(n):
            if u != v and (directed or u < v) and rng.random() < 0.45:
                eu.append(u)
                ev.append(v)
    mk = gg.from_edges_directed if directed else gg.from_edges
    g = mk(n, np.array(eu, np.int32), np.array(ev, np.int32))
    w = gg.edge_lengths(g, 1, 3, 61 + seed, symmetric=not directed)  # small range: many ties
    adj = [[(int(g.col[j]), int(w[j])) for j in range(g.row_ptr[u], g.row_ptr[u + 1])] for u in range(n)]
    for s in range(n):
        ref = [float(x) for x in _brute_delta_w(n, adj, s)]
        delta, _, _, _, _, _ = oracle.dependencies_w(g, w, s)
        assert rel_close(delta, ref, 1e-13), (seed, s)


def test_scaling_every_length_changes_nothing_but_distances():
    g = gg.rmat(9, 8, 0.57, 0.19, 0.19, 62)
    w = gg.edge_lengths(g, 1, 5, 63)
    for s in [0, 3, 100]:
        d1, dist1, sig1, o1, _, _ = oracle.dependencies_w(g, w, s)
        d3, dist3, sig3, o3, _, _ = oracle.dependencies_w(g, 3 * w, s)
        assert o1 == o3
        assert np.array_equal(d1, d3) and np.array_equal(sig1, sig3)
        assert np.array_equal(dist3, np.where(dist1 >= 0, 3 * dist1, -1))


@pytest.mark.parametrize("side", [20, 45])
def test_equal_length_grid_counts_are_binomials(side):
    # every edge of length 2: from the corner, sigma to (i, j) is C(i+j, i); on
    # the 45x45 grid C(88, 44) > 2^64, so the sample is in the extended form,
    # and its dependencies equal the unit-length grid's
    g = gg.grid(side)
    w = np.full(g.col.shape[0], 2, np.uint32)
    delta, dist, sig, ovf, sm, se = oracle.dependencies_w(g, w, 0)
    assert ovf == (math.comb(2 * side - 2, side - 1) >= 2**64)
    for v in range(g.n):
        i, j = divmod(v, side)
        assert dist[v] == 2 * (i + j)
        exact = math.comb(i + j, i)
        got = Fraction(sm[v]) * Fraction(2) ** int(se[v])
        if exact < 2**53:
            assert got == exact
        else:
            assert abs(got - exact) <= Fraction(exact) * Fraction(1.01 * (i + j) * U)
    d1, _, _, _ = oracle.dependencies(g, 0)
    assert np.array_equal(delta, d1)


def _wgraph(n, edges):
    """Undirected graph from (u, v, length) triples: CSR rows sorted, lengths
    on both rows."""
    adj = [dict() for _ in range(n)]
    for u, v, k in edges:
        adj[u][v] = k
        adj[v][u] = k
    rp = np.zeros(n + 1, np.int32)
    col, w = [], []
    for u in range(n):
        for v in sorted(adj[u]):
            col.append(v)
            w.append(adj[u][v])
        rp[u + 1] = len(col)
    g = gg.from_edges(n, np.array([e[0] for e in edges], np.int32), np.array([e[1] for e in edges], np.int32))
    assert np.array_equal(g.row_ptr, rp) and np.array_equal(g.col, np.array(col, np.int32))
    return g, np.array(w, np.uint32)


@pytest.mark.parametrize("long_side,bc_b", [(3, 2.0), (2, 1.0), (1, 0.0)])
def test_weighted_triangle_closed_forms(long_side, bc_b):
    # a-b and b-c of length 1, a-c of length L: for L = 3 both ordered pairs
    # (a,c), (c,a) go through b (BC(b) = 2); for L = 2 the direct edge ties the
    # path through b (each pair splits 1/2, BC(b) = 1); for L = 1 the direct
    # edge wins (BC(b) = 0). Ordered pairs, R1.
    g, w = _wgraph(3, [(0, 1, 1), (1, 2, 1), (0, 2, long_side)])
    bc = oracle.exact_bc_w(g, w)
    assert bc[1] == bc_b and bc[0] == 0.0 and bc[2] == 0.0
    _, dist, sig, _, _, _ = oracle.dependencies_w(g, w, 0)
    assert dist.tolist() == [0, 1, min(2, long_side)]
    assert sig[2] == (2 if long_side == 2 else 1)


def test_weighted_square_with_unequal_sides():
    # the 4-cycle a-b-c-d-a with lengths ab = 1, bc = 1, cd = 2, da = 2:
    # a to c is 2 through b (through d it is 4), so b carries (a,c) and (c,a);
    # b to d is 3 both through a and through c, so a and c each carry half of
    # (b,d) and of (d,b); every other pair is an edge that is a shortest path.
    g, w = _wgraph(4, [(0, 1, 1), (1, 2, 1), (2, 3, 2), (3, 0, 2)])
    bc = oracle.exact_bc_w(g, w)
    assert bc.tolist() == [1.0, 2.0, 1.0, 0.0]
    assert math.isclose(float(np.sum(bc)), 4.0)


def test_edge_length_generator():
    # inputs, not arithmetic of the method: both rows of an undirected edge get
    # the same length, lengths stay in [lo, hi], cover it, and repeat per seed
    g = gg.erdos_renyi(500, 6, 95)
    w = gg.edge_lengths(g, 3, 9, 96)
    assert w.dtype == np.uint32 and w.shape == g.col.shape
    assert w.min() == 3 and w.max() == 9
    pos = {}
    for u in range(g.n):
        for j in range(g.row_ptr[u], g.row_ptr[u + 1]):
            pos[(u, int(g.col[j]))] = int(w[j])
    assert all(pos[(v, u)] == k for (u, v), k in pos.items())
    assert np.array_equal(w, gg.edge_lengths(g, 3, 9, 96))
    assert not np.array_equal(w, gg.edge_lengths(g, 3, 9, 97))
    d = gg.directed_er(500, 6, 98)
    wd = gg.edge_lengths(d, 1, 1000, 99, symmetric=False)
    assert wd.min() >= 1 and wd.max() <= 1000 and len(np.unique(wd)) > 900
    with pytest.raises(ValueError):
        gg.edge_lengths(g, 0, 5, 1)
