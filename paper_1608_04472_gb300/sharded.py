"""One query shared by G ranks (one GPU each): block assignment and exchange.

The draws of a query are independent (Sec. 4 step 2; Algorithm 1), so the
draw sequence is cut into blocks of B draws dealt round-robin: in round r,
rank q computes block r*G + q. After each round the ranks allgather their
blocks of per-draw target values and every rank runs the same stop scan over
the G blocks in draw order (``bc_scan_block``, the arithmetic of Sec. 4 step 3
and of Algorithm 1's loop test), so the stop counts, sums and estimates are
those of one GPU, whatever G and B. At most G*B - 1 draws past the last stop
are computed. For the uniform all-vertex estimate each rank adds the exact
sums of its blocks (``bc_uniform_partial``: 32-bit chunks in int64), one
integer allreduce adds the ranks' partials, and ``bc_acc_estimate`` rounds
once: bit-identical to one GPU as well.

The collectives are passed in as callables (``allgather(ndarray) -> list of
ndarrays`` in rank order, ``allreduce_sum(int64 ndarray) -> ndarray``), so the
same code runs over NCCL on GPUs and over gloo on CPU; ``torch_collectives``
builds them from ``torch.distributed``. This module only deals out blocks and
moves arrays: every value comes from the library's entry points.
"""
from __future__ import annotations

import numpy as np

from . import capi


def adaptive_sharded(block_fn, T: int, n_scale: float, cn: float, cap: int, rank: int, world: int, allgather,
                     B: int = 256, threshold_scale: float = 1.0) -> dict:
    """The adaptive loop over draws 0 .. cap-1 shared by `world` ranks.
    block_fn(i0, count) -> float64 [T][count]: the per-draw values of draws
    i0 .. i0+count-1 (this rank's block). Returns k, S, status, est of the T
    targets (the same on every rank)."""
    S = np.zeros(T, np.float64)
    k = np.zeros(T, np.int64)
    done = np.zeros(T, np.int32)
    est = np.zeros(T, np.float64)
    status = np.ones(T, np.int32)
    state = (S, k, done, est, status)
    remaining = T
    base = 0
    while remaining > 0 and base < cap:
        i0 = base + rank * B
        cnt = max(0, min(B, cap - i0))
        mine = np.zeros((T, B), np.float64)
        if cnt > 0:
            mine[:, :cnt] = block_fn(i0, cnt)
        blocks = allgather(mine)
        for q in range(world):
            j0 = base + q * B
            c = max(0, min(B, cap - j0))
            if c == 0 or remaining == 0:
                break
            remaining = capi.bc_scan_block(blocks[q][:, :c], j0, cn, threshold_scale, n_scale, state)
        base += world * B
    return {"k": k, "S": S, "status": status, "est": est}


def uniform_sharded(partial_fn, n: int, k: int, rank: int, world: int, allreduce_sum, B: int = 1024) -> np.ndarray:
    """The uniform estimate over draws 0 .. k-1 shared by `world` ranks.
    partial_fn(i0, count, parts) adds the exact sums of draws i0 .. i0+count-1
    into parts (int64 [n][6])."""
    parts = np.zeros((n, 6), np.int64)
    for i0 in range(rank * B, k, world * B):
        partial_fn(i0, min(B, k - i0), parts)
    parts = np.ascontiguousarray(allreduce_sum(parts), dtype=np.int64)
    return capi.bc_acc_estimate(parts, k)


def adaptive_sources_sharded(ctx, g: int, targets, c: float, cap: int, seed: int, qid: int, rank: int, world: int,
                             allgather, B: int = 256) -> dict:
    """bc_adaptive_sources' results for one query computed by `world` ranks."""
    n, _ = capi.bc_graph_info(ctx.ptr, g)
    t = np.ascontiguousarray(targets, dtype=np.int32)
    return adaptive_sharded(lambda i0, cnt: ctx.target_dependencies(g, t, seed, qid, i0, cnt), t.size, float(n),
                            c * n, cap, rank, world, allgather, B)


def adaptive_pairs_sharded(ctx, g: int, targets, c: float, cap: int, seed: int, qid: int, rank: int, world: int,
                           allgather, B: int = 256, threshold_scale: float = 1.0) -> dict:
    """bc_adaptive_pairs' results for one query computed by `world` ranks
    (each rank's blocks from bc_pair_values, which keeps the target BFSs of
    the query between its blocks)."""
    n, _ = capi.bc_graph_info(ctx.ptr, g)
    t = np.ascontiguousarray(targets, dtype=np.int32)
    return adaptive_sharded(lambda i0, cnt: ctx.pair_values(g, t, seed, qid, i0, cnt), t.size,
                            float(n) * float(n - 1), c * n, cap, rank, world, allgather, B, threshold_scale)


def uniform_sources_sharded(ctx, g: int, k: int, seed: int, qid: int, rank: int, world: int, allreduce_sum,
                            B: int = 1024) -> np.ndarray:
    """bc_uniform_sources' estimate for one query computed by `world` ranks."""
    n, _ = capi.bc_graph_info(ctx.ptr, g)
    return uniform_sharded(lambda i0, cnt, parts: ctx.uniform_partial(g, seed, qid, i0, cnt, parts), n, k, rank,
                           world, allreduce_sum, B)


def torch_collectives(dist, device, group=None):
    """(allgather, allreduce_sum) over a torch.distributed process group; arrays
    travel as tensors on `device` ("cuda" for NCCL, "cpu" for gloo)."""
    import torch

    world = dist.get_world_size(group)

    def allgather(a: np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(a)).to(device)
        outs = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(outs, t, group=group)
        return [o.cpu().numpy() for o in outs]

    def allreduce_sum(a: np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(a)).to(device)
        dist.all_reduce(t, group=group)
        return t.cpu().numpy()

    return allgather, allreduce_sum
