"""The identity behind the bidirectional pair search, checked with the
oracle's own BFS counts: for an undirected graph and reachable s != t with
d = d(s,t), every level a in [0, d] is a cut of the shortest s-t paths, so
    sigma_st = sum over x with d(s,x) = a and d(x,t) = d - a of sigma_sx * sigma_xt,
and no vertex x has d(s,x) + d(x,t) < d. The kernel meets at one such level
(where the two balls first touch); any level must give the same count."""
import numpy as np
import pytest

import graphgen as gg
import oracle


@pytest.mark.parametrize("make", [
    lambda: gg.barabasi_albert(400, 3, 21),
    lambda: gg.erdos_renyi(300, 2.5, 22),  # several components: unreachable pairs
    lambda: gg.grid(12),
    lambda: gg.rmat(8, 6, 0.57, 0.19, 0.19, 23),
])
def test_every_level_is_a_cut_of_the_shortest_paths(make):
    g = make()
    rng = np.random.default_rng(5)
    bfs = {}

    def row(v):
        if v not in bfs:
            _, dist, sig, ovf = oracle.dependencies(g, v)
            assert not ovf
            bfs[v] = (dist.astype(np.int64), sig.astype(object))
        return bfs[v]

    for _ in range(40):
        s, t = (int(x) for x in rng.integers(0, g.n, 2))
        if s == t:
            continue
        ds, ss = row(s)
        dt, st = row(t)
        d = int(ds[t])
        if d < 0:
            assert dt[s] < 0  # undirected: unreachable both ways
            continue
        assert dt[s] == d and ss[t] == st[s]
        both = (ds >= 0) & (dt >= 0)
        assert np.all(ds[both] + dt[both] >= d)
        for a in range(d + 1):
            on = np.nonzero(both & (ds == a) & (dt == d - a))[0]
            assert sum(ss[x] * st[x] for x in on) == ss[t], (s, t, a)
