"""Pins for the oracle on directed graphs (paths follow the edges' direction;
BC over ordered pairs, Def. 1): networkx's directed betweenness (no halving
for directed graphs), brute-force enumeration of every directed shortest path
on small graphs, the dependency-sum invariant, and binomial path counts on a
grid whose edges point right and down, including counts beyond 2^64 (the
extended form pulls over in-neighbours)."""
import math
from fractions import Fraction

import networkx as nx
import numpy as np
import pytest

import graphgen as gg
import oracle
from test_oracle_pins import rel_close

U = 2.0**-53


def _nx_digraph(g):
    G = nx.DiGraph()
    G.add_nodes_from(range(g.n))
    for u in range(g.n):
        for w in g.col[g.row_ptr[u]:g.row_ptr[u + 1]].tolist():
            G.add_edge(u, w)
    return G


@pytest.mark.parametrize("make", [lambda: gg.directed_er(300, 3, 5), lambda: gg.directed_rmat(9, 8, 0.57, 0.19, 0.19, 6)])
def test_directed_bc_matches_networkx(make):
    g = make()
    ref = nx.betweenness_centrality(_nx_digraph(g), normalized=False)
    bc = oracle.exact_bc(g)
    assert rel_close(bc, [ref[v] for v in range(g.n)], 1e-9)


def _brute_delta(g, s):
    """delta_s(v) from every directed shortest path out of s (exact rationals)."""
    out = [g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist() for v in range(g.n)]
    paths = {}

    def dfs(path, seen):
        v = path[-1]
        paths.setdefault(v, []).append(tuple(path))
        for w in out[v]:
            if w not in seen:
                seen.add(w)
                path.append(w)
                dfs(path, seen)
                path.pop()
                seen.discard(w)

    dfs([s], {s})
    delta = [Fraction(0)] * g.n
    for t, ps in paths.items():
        if t == s:
            continue
        L = min(len(p) for p in ps)
        sp = [p for p in ps if len(p) == L]
        for v in range(g.n):
            if v not in (s, t):
                k = sum(1 for p in sp if v in p)
                if k:
                    delta[v] += Fraction(k, len(sp))
    return delta


@pytest.mark.parametrize("seed", range(10))
def test_directed_bruteforce_small(seed):
    n = 5 + seed % 4
    rng = np.random.default_rng(200 + seed)
    eu, ev = np.nonzero(rng.random((n, n)) < 0.35)
    g = gg.from_edges_directed(n, eu, ev)
    for s in range(n):
        ref = [float(x) for x in _brute_delta(g, s)]
        delta, _, _, _ = oracle.dependencies(g, s)
        assert rel_close(delta, ref, 1e-13), (seed, s)
        dx, _, _, _ = oracle.dependencies_xf(g, s)
        assert rel_close(dx, ref, 1e-13), (seed, s)


def test_directed_dependency_sum_invariant():
    g = gg.directed_rmat(10, 8, 0.57, 0.19, 0.19, 7)
    for s in [0, 1, 17, g.n - 1]:
        delta, dist, _, _ = oracle.dependencies(g, s)
        expect = float(np.sum(dist[dist > 0] - 1))
        assert math.isclose(math.fsum(delta), expect, rel_tol=1e-12, abs_tol=1e-9)


@pytest.mark.parametrize("side", [20, 45])
def test_directed_grid_counts_are_binomials(side):
    # from the corner every vertex (i, j) is reached by C(i+j, i) paths; a 45x45
    # corner count C(88, 44) exceeds 2^64, so that sample is in the extended form
    g = gg.directed_grid(side)
    delta, dist, sm, se = oracle.dependencies_xf(g, 0)
    for v in range(g.n):
        i, j = divmod(v, side)
        assert dist[v] == i + j
        exact = math.comb(i + j, i)
        got = Fraction(sm[v]) * Fraction(2) ** int(se[v])
        if exact < 2**53:
            assert got == exact
        else:
            assert abs(got - exact) <= Fraction(exact) * Fraction(1.01 * (i + j) * U)
    d2, _, _, ovf = oracle.dependencies(g, 0)
    assert ovf == (math.comb(2 * side - 2, side - 1) >= 2**64)
    if ovf:
        assert np.array_equal(d2, delta)
    # every s-t shortest path has d(s,t) - 1 interior vertices
    expect = sum(d - 1 for d in dist.tolist() if d > 0)
    assert math.isclose(math.fsum(delta), expect, rel_tol=1e-9)
