"""The GPU side of one query shared by several ranks: bc_target_dependencies
blocks, bc_pair_values blocks and bc_uniform_partial partials computed on the
GPU, combined by the sharding driver (rank partials summed as integers, blocks
scanned in draw order), must give bc_adaptive_sources', bc_adaptive_pairs' and
bc_uniform_sources' results bit for bit, for any block size; the blocks
themselves equal the oracle's per-draw target dependencies and pair values. (The exchange between processes is covered on CPU by
tests/test_sharded_cpu.py.)"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1608_04472_gb300 as pkg
    c = pkg.Context(0, batch_width=64)
    yield c
    c.close()


@pytest.mark.parametrize("family", ["er2000", "rmat_s14_hubs"])
def test_sharded_matches_single_gpu(ctx, family):
    from paper_1608_04472_gb300 import sharded
    g = {"er2000": lambda: gg.erdos_renyi(2000, 8, 1),
         "rmat_s14_hubs": lambda: gg.rmat(14, 16, 0.57, 0.19, 0.19, 7)}[family]()
    targets = np.concatenate([gg.uniform_targets(g.n, 12, 3),
                              np.argsort(-g.degrees(), kind="stable")[:4]]).astype(np.int32)
    targets = np.unique(targets)
    c, cap, seed, qid = 3.0, 3000, 11, 5
    h = ctx.load_graph(g.row_ptr, g.col)
    try:
        ref = ctx.adaptive_sources(h, targets, c, cap, seed, qid)
        assert np.any(ref["status"] == 0) and np.any(ref["status"] == 1)
        for B in (64, 100, 1024):
            got = sharded.adaptive_sources_sharded(ctx, h, targets, c, cap, seed, qid, 0, 1, lambda a: [a], B)
            for key in ("k", "S", "status", "est"):
                assert np.array_equal(got[key], ref[key]), (B, key)
        # a block against the oracle's per-draw dependencies at the targets
        blk = ctx.target_dependencies(h, targets, seed, qid, 37, 70)
        for i in (0, 1, 69):
            s = oracle.draw_source(seed, qid, 37 + i, g.n)
            assert np.array_equal(blk[:, i], oracle.dependencies(g, s)[0][targets]), i
        # the uniform estimate from three ranks' partials, summed as integers
        k = 1500
        uni = ctx.uniform_sources(h, k, seed, qid + 1)
        for B in (128, 1024):
            parts = [np.zeros((g.n, 6), np.int64) for _ in range(3)]
            for r in range(3):
                for i0 in range(r * B, k, 3 * B):
                    ctx.uniform_partial(h, seed, qid + 1, i0, min(B, k - i0), parts[r])
            est = sharded.uniform_sharded(lambda i0, cnt, p: None, g.n, k, 0, 1, lambda a: parts[0] + parts[1] + parts[2])
            assert np.array_equal(est, uni), B
    finally:
        ctx.free_graph(h)


@pytest.mark.parametrize("family", ["er3000", "ba20000"])
def test_sharded_pairs_match_single_gpu(ctx, family):
    from paper_1608_04472_gb300 import sharded
    g = {"er3000": lambda: gg.erdos_renyi(3000, 8, 2),
         "ba20000": lambda: gg.barabasi_albert(20000, 4, 3)}[family]()
    targets = np.unique(np.concatenate([gg.uniform_targets(g.n, 6, 4),
                                        np.argsort(-g.degrees(), kind="stable")[:3]])).astype(np.int32)
    c, cap, seed, qid, scale = 1.0, 2500, 13, 9, 500.0
    h = ctx.load_graph(g.row_ptr, g.col)
    try:
        ref = ctx.adaptive_pairs(h, targets, c, cap, seed, qid, scale)
        assert np.any(ref["status"] == 0) and np.any(ref["status"] == 1)
        for B in (64, 300):
            got = sharded.adaptive_pairs_sharded(ctx, h, targets, c, cap, seed, qid, 0, 1, lambda a: [a], B,
                                                 scale)
            for key in ("k", "S", "status", "est"):
                assert np.array_equal(got[key], ref[key]), (B, key)
        # rank 0's view with three ranks: every rank's blocks computed here and
        # handed out round by round, as the allgather would
        ranks, B = 3, 200
        rounds = (cap + ranks * B - 1) // (ranks * B)
        blocks = {}
        for r in range(ranks):
            for rnd in range(rounds):
                i0 = rnd * ranks * B + r * B
                cnt = max(0, min(B, cap - i0))
                blk = np.zeros((targets.size, B))
                if cnt:
                    blk[:, :cnt] = ctx.pair_values(h, targets, seed, qid, i0, cnt)
                blocks[(r, rnd)] = blk
        served = [0]

        def allgather(a):
            out = [blocks[(r, served[0])] for r in range(ranks)]
            served[0] += 1
            return out
        res = sharded.adaptive_sharded(lambda i0, cnt: blocks[(0, i0 // (ranks * B))][:, :cnt], targets.size,
                                       float(g.n) * float(g.n - 1), c * g.n, cap, 0, ranks, allgather, B, scale)
        for key in ("k", "S", "status", "est"):
            assert np.array_equal(res[key], ref[key]), key
        # a block against the oracle's per-draw pair values
        blk = ctx.pair_values(h, targets, seed, qid, 1000, 129)
        want = oracle.pair_sequence_multi(g, targets, seed, qid, 1000, 129)
        np.testing.assert_array_equal(blk, want)
        # another target set on the same graph replaces the cached tables
        other = targets[::-1].copy()
        np.testing.assert_array_equal(ctx.pair_values(h, other, seed, qid, 1000, 129), want[::-1])
    finally:
        ctx.free_graph(h)
