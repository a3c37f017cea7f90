"""Hand-derived fixtures (tests/golden/hand_examples.txt): BC per Def. 1 and
per-source dist/sigma/delta per Def. 2-3, checked against the CPU oracle."""
import os

import numpy as np

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.txt")


def load_cases():
    cases = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, n, edges, bc, src, dist, sigma, delta = [x.strip() for x in line.split("|")]
        e = [tuple(int(x) for x in pair.split("-")) for pair in edges.split()]
        cases.append(dict(name=name, n=int(n), edges=e,
                          bc=[float(x) for x in bc.split()], src=int(src),
                          dist=[int(x) for x in dist.split()],
                          sigma=[int(x) for x in sigma.split()],
                          delta=[float(x) for x in delta.split()]))
    return cases


def test_hand_examples():
    cases = load_cases()
    assert len(cases) == 2
    for c in cases:
        e = np.array(c["edges"], np.int32)
        g = gg.from_edges(c["n"], e[:, 0], e[:, 1], c["name"])
        assert oracle.exact_bc(g).tolist() == c["bc"], c["name"]
        delta, dist, sigma, _ = oracle.dependencies(g, c["src"])
        assert dist.tolist() == c["dist"]
        assert sigma.tolist() == c["sigma"]
        assert delta.tolist() == c["delta"]
