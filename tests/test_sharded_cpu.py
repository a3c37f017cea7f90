"""One query shared by two gloo ranks on CPU (paper_1608_04472_gb300/sharded.py):
the per-block values come from the oracle inside the test (what each rank's GPU
computes with bc_target_dependencies / bc_uniform_partial), the exchange runs
over gloo, and the combination goes through the library's host calls
(bc_scan_block, bc_acc_add_rows, bc_acc_estimate). Bader's and Algorithm 1's
k, S, status and est and the uniform estimate must be identical at G = 1 and
G = 2, for several block sizes, and equal to the oracle's own single-threaded
runs."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

N_ER, DEG, GSEED = 300, 6, 5
TARGETS = [0, 7, 150, 299, 42, 123]
C, CAP, SEED, QID = 1.5, 300, 21, 3
K_UNI = 90
PC, PCAP, PSCALE = 1.2, 400, 150.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run(rank, world, allgather, allreduce_sum, B):
    import graphgen as gg
    import oracle
    from paper_1608_04472_gb300 import capi, sharded

    g = gg.erdos_renyi(N_ER, DEG, GSEED)
    t = np.array(TARGETS, np.int32)

    def block_fn(i0, cnt):
        rows = [oracle.dependencies(g, oracle.draw_source(SEED, QID, i, g.n))[0][t] for i in range(i0, i0 + cnt)]
        return np.stack(rows, axis=1)

    def partial_fn(i0, cnt, parts):
        rows = np.stack([oracle.dependencies(g, oracle.draw_source(SEED, QID + 1, i, g.n))[0]
                         for i in range(i0, i0 + cnt)])
        capi.bc_acc_add_rows(rows, parts)

    res = sharded.adaptive_sharded(block_fn, t.size, float(g.n), C * g.n, CAP, rank, world, allgather, B)
    est = sharded.uniform_sharded(partial_fn, g.n, K_UNI, rank, world, allreduce_sum, B)
    pairs = sharded.adaptive_sharded(lambda i0, cnt: oracle.pair_sequence_multi(g, t, SEED, QID + 2, i0, cnt),
                                     t.size, float(g.n) * float(g.n - 1), PC * g.n, PCAP, rank, world, allgather, B,
                                     PSCALE)
    return res, est, pairs


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1608_04472_gb300 import sharded
    ag, ar = sharded.torch_collectives(dist, "cpu")
    out = {}
    for B in (16, 64, 1024):
        out[B] = _run(rank, world, ag, ar, B)
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def _single(B):
    return _run(0, 1, lambda a: [a], lambda a: a, B)


def test_two_ranks_match_one_rank_and_the_oracle():
    import graphgen as gg
    import oracle
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = gg.erdos_renyi(N_ER, DEG, GSEED)
    ref = oracle.adaptive_sources(g, TARGETS, C, CAP, SEED, QID)
    ref_u = oracle.uniform_sources(g, K_UNI, SEED, QID + 1)
    ref_p = oracle.adaptive_pairs(g, TARGETS, PC, PCAP, SEED, QID + 2, PSCALE)
    assert np.any(ref["status"] == oracle.STOPPED) and np.any(ref["status"] == oracle.CAPPED)
    assert np.any(ref_p["status"] == oracle.STOPPED) and np.any(ref_p["status"] == oracle.CAPPED)
    for B in (16, 64, 1024):
        one, est1, p1 = _single(B)
        for rank in range(world):
            two, est2, p2 = res[rank][B]
            for key in ("k", "S", "status", "est"):
                assert np.array_equal(two[key], one[key]), (B, rank, key)
                assert np.array_equal(one[key], ref[key]), (B, key)
                assert np.array_equal(p2[key], p1[key]), (B, rank, "pairs", key)
                assert np.array_equal(p1[key], ref_p[key]), (B, "pairs", key)
            assert np.array_equal(est2, est1) and np.array_equal(est1, ref_u), B


def test_exact_chunks_round_like_the_oracle():
    """bc_acc_add_rows + bc_acc_estimate against the oracle's exact sum of the
    same rows, including values at the ends of the exact window."""
    import oracle
    from paper_1608_04472_gb300 import capi
    rng = np.random.default_rng(3)
    n, k = 64, 40
    rows = np.ldexp(rng.random((k, n)) + 0.5, rng.integers(-70, 60, size=(k, n)))
    rows[rng.random((k, n)) < 0.2] = 0.0
    rows[0, :4] = [2.0 ** -76, 2.0 ** 62 * 1.9, 1.0, 3.0]
    parts = np.zeros((n, 6), np.int64)
    capi.bc_acc_add_rows(rows[:17], parts)
    capi.bc_acc_add_rows(rows[17:], parts)
    est = capi.bc_acc_estimate(parts, k)
    for v in range(n):
        S = oracle.exact_sum(rows[:, v])
        assert est[v] == (n * S) / k, v
    with pytest.raises(capi.BCError):
        capi.bc_acc_add_rows(np.full((1, n), 2.0 ** 63), np.zeros((n, 6), np.int64))
