"""The oracle's steps for parallel drivers, pinned to the pinned oracle calls.

UniformAccumulator fed with rows in any order and by vertex ranges must give
uniform_sources bit for bit (the sums are exact); pair_sequence_multi must give
pair_sequence for each target; the stop-rule replays used at full size must
reproduce adaptive_sources / adaptive_pairs (k, S, status, est) exactly,
including capped targets, on graphs small enough for the plain oracle calls.
"""
import numpy as np

import graphgen as gg
import oracle
from tests import _oracle_par as par


def test_accumulator_matches_uniform_sources_in_any_order():
    g = gg.erdos_renyi(400, 5, 3)
    k, seed, qid = 57, 4, 11
    srcs = [oracle.draw_source(seed, qid, i, g.n) for i in range(k)]
    rows = np.stack([oracle.dependencies(g, s)[0] for s in srcs])
    acc = oracle.UniformAccumulator(g.n)
    perm = np.random.default_rng(1).permutation(k)
    acc.add_rows(rows[perm[:20]], 0, 150)
    acc.add_rows(rows[perm[:20]], 150, g.n)
    for i in perm[20:]:
        acc.add_rows(rows[i:i + 1], 0, 399)
        acc.add_rows(rows[i:i + 1], 399, g.n)
    assert np.array_equal(acc.estimate(k), oracle.uniform_sources(g, k, seed, qid))
    acc.close()


def test_parallel_uniform_estimate_matches_uniform_sources():
    g = gg.rmat(10, 8, 0.57, 0.19, 0.19, 5)
    k, seed, qid = 150, 9, 2
    srcs = [oracle.draw_source(seed, qid, i, g.n) for i in range(k)]
    seen = []
    est = par.uniform_estimate(g, srcs, chunk=32, on_rows=lambda i0, r: seen.append((i0, r.shape[0])))
    assert np.array_equal(est, oracle.uniform_sources(g, k, seed, qid))
    assert sum(c for _, c in seen) == k and [i for i, _ in seen] == list(range(0, k, 32))


def test_pair_sequence_multi_matches_single_target_sequences():
    g = gg.barabasi_albert(500, 3, 7)
    targets = np.array([0, 3, 250, 499], np.int32)
    y = oracle.pair_sequence_multi(g, targets, 5, 6, 10, 90)
    for j, v in enumerate(targets):
        y1, _, _ = oracle.pair_sequence(g, int(v), 5, 6, 10, 90)
        assert np.array_equal(y[j], y1)


def test_pair_sequence_multi_extended_counts():
    """A 70x70 grid: the corner targets' counts and many sigma_st exceed 2^64."""
    g = gg.grid(70)
    targets = np.array([0, 35 * 70 + 35, 70 * 70 - 1], np.int32)
    y = oracle.pair_sequence_multi(g, targets, 8, 1, 0, 12)
    for j, v in enumerate(targets):
        assert np.array_equal(y[j], oracle.pair_sequence(g, int(v), 8, 1, 0, 12)[0])


def test_bader_replay_matches_adaptive_sources():
    g = gg.erdos_renyi(300, 6, 5)
    targets = np.array([0, 7, 150, 299, 42], np.int32)
    for c, cap in [(1.5, 400), (3.0, 40)]:  # some targets stop, some reach the cap
        res = oracle.adaptive_sources(g, targets, c, cap, 21, 3)
        srcs = [oracle.draw_source(21, 3, i, g.n) for i in range(cap)]
        X = par.target_columns(g, srcs, targets)
        k, S, st, est = par.replay_bader(X, g.n, c, cap)
        assert np.array_equal(k, res["k"]) and np.array_equal(S, res["S"])
        assert np.array_equal(st, res["status"]) and np.array_equal(est, res["est"])
    assert np.any(res["status"] == oracle.CAPPED)


def test_pair_replay_matches_adaptive_pairs():
    g = gg.erdos_renyi(60, 4, 8)
    targets = np.array([3, 30, 59], np.int32)
    for scale in [1.0, float(g.n - 1)]:
        res = oracle.adaptive_pairs(g, targets, 1.0, 800, 4, 9, threshold_scale=scale)
        Y = par.pair_values(g, targets, 4, 9, 800)
        k, S, st, est = par.replay_pairs(Y, g.n, 1.0, 800, scale)
        assert np.array_equal(k, res["k"]) and np.array_equal(S, res["S"])
        assert np.array_equal(st, res["status"]) and np.array_equal(est, res["est"])
