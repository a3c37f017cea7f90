"""Pins for the oracle's extended form: samples whose shortest-path counts
exceed 2^64-1 are recomputed with doubles of unbounded exponent (m * 2^e).

The pins are independent of the oracle's arithmetic:
  * one extended addition against Python's exact rationals, rounded to 53 bits
    by int/int true division (correctly rounded in CPython);
  * path counts from a grid corner against binomial coefficients (exact ints),
    within the bound of one rounding per level, and equal where they are
    below 2^53;
  * dependencies against a 60-digit decimal evaluation of Theorem 1 on exact
    integer counts, within a bound derived from the number of roundings;
  * dependencies on trees (every count 1) against subtree sizes, exactly;
  * dependencies against brute-force path enumeration on small graphs;
  * the invariant sum_v delta_s(v) = sum_t (d(s,t) - 1).
"""
import decimal
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle
from test_oracle_pins import brute_bc_and_delta, graph_from_edges, rel_close

U = 2.0**-53


def _rn_unbounded(x: Fraction):
    """x > 0 rounded to 53 bits with no exponent limit -> (m in [1,2), e)."""
    E = x.numerator.bit_length() - x.denominator.bit_length()
    if Fraction(2) ** E > x:
        E -= 1
    scaled = x / (Fraction(2) ** E)  # in [1, 2)
    m = scaled.numerator / scaled.denominator  # correctly rounded
    if m == 2.0:
        m, E = 1.0, E + 1
    return m, E


def _xf_value(m, e):
    return Fraction(m) * Fraction(2) ** e


def test_xf_add_correctly_rounded_random():
    rng = random.Random(5)
    for _ in range(4000):
        m1 = 1.0 + rng.random()
        m2 = 1.0 + rng.random()
        e1 = rng.randint(-3000, 3000)
        e2 = e1 + rng.randint(-70, 70)
        got = oracle.xf_add(m1, e1, m2, e2)
        assert got == _rn_unbounded(_xf_value(m1, e1) + _xf_value(m2, e2)), (m1, e1, m2, e2)


def test_xf_add_ties_and_zero():
    # 1 + 2^-53 is a tie: to even (1.0); a hair above the tie rounds up
    assert oracle.xf_add(1.0, 0, 1.0, -53) == (1.0, 0)
    assert oracle.xf_add(1.0, 0, 1.0 + 2.0**-52, -53) == (1.0 + 2.0**-52, 0)
    # (1 + 2^-52) + 2^-53 is a tie with an odd last bit: up to even
    assert oracle.xf_add(1.0 + 2.0**-52, 700, 1.0, 647) == (1.0 + 2.0**-51, 700)
    # carry into the next binade, far outside the double range
    assert oracle.xf_add(1.5, 5000, 1.5, 5000) == (1.5, 5001)
    assert oracle.xf_add(0.0, 0, 1.25, -4000) == (1.25, -4000)
    # a term 61 binades down is below a quarter ulp
    assert oracle.xf_add(1.0, 0, 1.999, -61) == (1.0, 0)


def _exact_counts(g, s):
    """BFS distances and exact integer path counts (Python ints)."""
    dist = [-1] * g.n
    sig = [0] * g.n
    dist[s], sig[s] = 0, 1
    frontier = [s]
    while frontier:
        nxt = []
        for v in frontier:
            for w in g.neighbors(v).tolist():
                if dist[w] < 0:
                    dist[w] = dist[v] + 1
                    nxt.append(w)
                if dist[w] == dist[v] + 1:
                    sig[w] += sig[v]
        frontier = nxt
    return dist, sig


def _decimal_delta(g, s, dist, sig):
    """Theorem 1 evaluated with 60-digit decimals on exact counts."""
    ctx = decimal.Context(prec=60)
    D = decimal.Decimal
    order = sorted((v for v in range(g.n) if dist[v] >= 0), key=lambda v: -dist[v])
    delta = [D(0)] * g.n
    for v in order:
        acc = D(0)
        for w in g.neighbors(v).tolist():
            if dist[w] == dist[v] + 1:
                acc = ctx.add(acc, ctx.multiply(ctx.divide(D(sig[v]), D(sig[w])), ctx.add(D(1), delta[w])))
        delta[v] = acc if v != s else D(0)
    return delta


@pytest.mark.parametrize("side,src", [(40, "corner"), (90, "centre"), (12, "corner")])
def test_grid_counts_against_binomials(side, src):
    g = gg.grid(side)
    s = 0 if src == "corner" else (side // 2) * side + side // 2
    si, sj = divmod(s, side)
    delta, dist, sm, se = oracle.dependencies_xf(g, s)
    for v in range(g.n):
        i, j = divmod(v, side)
        a, b = abs(i - si), abs(j - sj)
        assert dist[v] == a + b
        exact = math.comb(a + b, a)
        got = _xf_value(sm[v], int(se[v]))
        if exact < 2**53:
            assert got == exact
        else:
            L = a + b
            assert abs(got - exact) <= Fraction(exact) * Fraction(1.01 * L * U), (v, got, exact)
    # the tiered call recomputes exactly the overflowing samples in this form
    d2, _, _, ovf = oracle.dependencies(g, s)
    biggest = max(math.comb(abs(i - si) + abs(j - sj), abs(i - si)) for i in range(side) for j in range(side))
    assert ovf == (biggest >= 2**64)
    if ovf:
        assert np.array_equal(d2, delta)


@pytest.mark.parametrize("side,s", [(36, 0), (36, 36 * 17 + 5), (14, 3)])
def test_grid_dependencies_against_decimal(side, s):
    g = gg.grid(side)
    dist, sig = _exact_counts(g, s)
    ref = _decimal_delta(g, s, dist, sig)
    delta, dist_x, _, _ = oracle.dependencies_xf(g, s)
    assert dist_x.tolist() == dist
    L = max(dist)
    tol = (L * (2 * L + 6) + 10) * U  # roundings along the deepest chain
    for v in range(g.n):
        r = float(ref[v])
        assert abs(delta[v] - r) <= tol * max(abs(r), 1.0), (v, delta[v], r)
    # invariant: every s-t shortest path has d(s,t) - 1 interior vertices
    expect = sum(d - 1 for d in dist if d > 0)
    assert math.isclose(math.fsum(delta), expect, rel_tol=tol)
    if max(sig) >= 2**64:
        d2, _, _, ovf = oracle.dependencies(g, s)
        assert ovf and np.array_equal(d2, delta)


def _random_tree(n, seed):
    rng = np.random.default_rng(seed)
    return graph_from_edges(n, [(int(rng.integers(0, v)), v) for v in range(1, n)])


@pytest.mark.parametrize("seed", range(4))
def test_tree_dependencies_are_subtree_sizes(seed):
    g = _random_tree(300, seed)
    for s in [0, 7, 299]:
        delta, dist, sm, se = oracle.dependencies_xf(g, s)
        assert np.all(sm[dist >= 0] == 1.0) and np.all(se == 0)
        # delta_s(v) = number of vertices strictly below v when the tree hangs from s
        below = [0] * g.n
        for v in sorted(range(g.n), key=lambda x: -dist[x]):
            for w in g.neighbors(v).tolist():
                if dist[w] == dist[v] + 1:
                    below[v] += below[w] + 1
        below[s] = 0
        assert delta.tolist() == [float(x) for x in below]


@pytest.mark.parametrize("seed", range(16))
def test_extended_form_against_bruteforce(seed):
    n = 4 + seed % 6
    rng = np.random.default_rng(100 + seed)
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.45]
    g = graph_from_edges(n, edges)
    _, delta_b = brute_bc_and_delta(g)
    for s in range(n):
        delta, _, _, _ = oracle.dependencies_xf(g, s)
        assert rel_close(delta, [float(x) for x in delta_b[s]], 1e-13)


def test_exact_bc_on_overflowing_grid_invariant():
    # every sample of a 36x36 grid from a corner region overflows; the total
    # over all sources still satisfies sum_v BC(v) = sum_{s != t} (d(s,t) - 1)
    side = 36
    g = gg.grid(side)
    bc = oracle.exact_bc(g)
    total = 0
    for a in range(side):
        for b in range(side):
            # ordered pairs at row offset a and column offset b
            cnt = (side - a) * (side - b) * (1 if a == 0 else 2) * (1 if b == 0 else 2)
            if a + b > 0:
                total += cnt * (a + b - 1)
    assert math.isclose(math.fsum(bc), total, rel_tol=1e-11)
    # symmetry of the grid: BC is invariant under the 8 symmetries of the square
    B = bc.reshape(side, side)
    assert np.allclose(B, B.T, rtol=1e-11) and np.allclose(B, B[::-1, :], rtol=1e-11)


def _grid_pair_exact(side, v, s, t):
    """sigma_sv sigma_vt / sigma_st on a grid from binomials (exact rational)."""
    (vi, vj), (si, sj), (ti, tj) = divmod(v, side), divmod(s, side), divmod(t, side)
    dst = abs(ti - si) + abs(tj - sj)
    dsv = abs(vi - si) + abs(vj - sj)
    dvt = abs(ti - vi) + abs(tj - vj)
    if v in (s, t) or dsv + dvt != dst:
        return Fraction(0)
    c = lambda a, b: math.comb(a + b, a)
    return Fraction(c(abs(vi - si), abs(vj - sj)) * c(abs(ti - vi), abs(tj - vj)), c(abs(ti - si), abs(tj - sj)))


@pytest.mark.parametrize("side", [40, 60])
def test_pair_values_on_overflowing_grid_against_binomials(side):
    # corner-to-corner counts C(2(side-1), side-1) exceed 2^64: the pair BFS and
    # (for central targets) the target BFS use the extended form
    g = gg.grid(side)
    rng = random.Random(side)
    s, t = 0, g.n - 1
    cases = [(rng.randrange(g.n), s, t) for _ in range(40)]
    cases += [((side // 2) * side + side // 2, s, t), (side + 1, s, t), (g.n - 2, s, t)]
    cases += [(rng.randrange(g.n), rng.randrange(g.n), rng.randrange(g.n)) for _ in range(40)]
    for v, a, b in cases:
        if a == b:
            continue
        exact = _grid_pair_exact(side, v, a, b)
        got = oracle.pair_value_of(g, v, a, b)
        if exact == 0:
            assert got == 0.0, (v, a, b)
        else:
            assert abs(Fraction(got) - exact) <= exact * Fraction(4 * 2 * side * U), (v, a, b, got, float(exact))


def test_pair_values_match_uint64_formula_where_counts_fit():
    # a 12x12 grid never overflows: the extended path is not taken and the value
    # is the plain double formula on exact counts
    g = gg.grid(12)
    for v, s, t in [(13, 0, 143), (50, 0, 143), (5, 3, 140), (77, 60, 80)]:
        exact = _grid_pair_exact(12, v, s, t)
        got = oracle.pair_value_of(g, v, s, t)
        assert abs(Fraction(got) - exact) <= exact * Fraction(2 * U)


def test_pair_sigma_st_extended_only_when_it_is_2_to_64_or_more():
    # R11 for pairs: the form of sigma_st depends on sigma_st alone. On a 90x90
    # grid from the corner, t = (14, 81) has sigma_st = C(95, 14), between 2^53
    # and 2^64, while counts in the middle of the same level, C(95, 47), exceed
    # 2^64. sigma_st is then the exact count rounded once, and the value is the
    # double formula on binomials; the pull-order extended sum of that count
    # differs from RN(C(95, 14)) in the last place, so the test tells the two
    # choices apart.
    side = 90
    g = gg.grid(side)
    ti, tj = 14, 81
    t = ti * side + tj
    c = math.comb(ti + tj, ti)
    assert 2**53 < c < 2**64 and math.comb(ti + tj, (ti + tj) // 2) >= 2**64
    _, _, sm, se = oracle.dependencies_xf(g, 0)
    assert Fraction(sm[t]) * Fraction(2) ** int(se[t]) != Fraction(float(c))
    for vi, vj in [(7, 40), (3, 20), (10, 60), (1, 1), (13, 80), (0, 5), (14, 2)]:
        a = float(math.comb(vi + vj, vi))
        b = float(math.comb(ti - vi + tj - vj, ti - vi))
        assert oracle.pair_value_of(g, vi * side + vj, 0, t) == (a * b) / float(c), (vi, vj)
    # and when sigma_st itself is beyond 2^64 the extended form is used: far corner
    far = g.n - 1
    exact = _grid_pair_exact(side, 45 * side + 45, 0, far)
    got = oracle.pair_value_of(g, 45 * side + 45, 0, far)
    assert abs(Fraction(got) - exact) <= exact * Fraction(4 * 2 * side * U)
