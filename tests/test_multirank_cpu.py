"""The multi-rank path of the benchmark on CPU: two gloo ranks run the same
per-rank plan and reductions bench.py uses under torchrun (one rank per GPU).
Ranks own disjoint query streams (weak scaling, no data-path collective); the
timed region is the max over ranks and samples are summed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    warm, timed = bench.rank_qids(rank, steps=3, warmup=2)
    # every qid of every rank, both streams (Bader q, uniform q+1)
    mine = [x for q in warm + timed for x in (q, q + 1)]
    allq = [None] * world
    dist.all_gather_object(allq, mine)
    ms, samples, edges = bench.reduce_over_ranks(dist, "cpu", 10.0 * (rank + 1), 100.0 + rank, 1e6)
    q.put((rank, allq, ms, samples, edges))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, allq, ms, samples, edges in res:
        flat = [x for per in allq for x in per]
        assert len(flat) == len(set(flat)), "ranks must not share draw streams"
        assert ms == 20.0  # max over ranks
        assert samples == 201.0 and edges == 2e6  # sums over ranks
