"""Multi-GPU multi-start GVNS: shard the starts over ranks, reduce the best.

Independent starts partition cleanly (Section 3's parallel scheme runs
searches side by side and keeps the minimum objective).  Rank r of N solves
the contiguous share of starts [lo_r, hi_r) on its own GPU with one
persistent launch and a device best-of; the only exchange is an all-reduce
(MIN) of one packed 64-bit key (cost << 24 | global start index), followed by
a broadcast of the winning solution from the rank that owns it.  Ties go to
the lowest start index, so the result equals the single-GPU best-of.

The collective layer is plain torch.distributed (NCCL on GPUs, gloo on CPU);
nothing of the method runs here.
"""
from __future__ import annotations

import numpy as np

KEY_COST_BITS = 40
KEY_INDEX_BITS = 24
INF_COST = (1 << KEY_COST_BITS) - 1
_KEY_BIAS = 1 << 63  # the unsigned 64-bit key, shifted into the int64 range


def pack_key(cost: int, start: int) -> int:
    """(cost, start) -> int64 key whose signed order is the lexicographic
    order of (cost, start): the unsigned key cost << 24 | start (INF -> all
    cost bits set) minus 2^63, so that every key, the INF sentinel included,
    fits a signed 64-bit MIN all-reduce."""
    if not 0 <= start < (1 << KEY_INDEX_BITS):
        raise ValueError("start index out of range")
    c = INF_COST if cost >= INF_COST else int(cost)
    if c < 0:
        raise ValueError("negative cost")
    return ((c << KEY_INDEX_BITS) | int(start)) - _KEY_BIAS


def unpack_key(key: int):
    u = int(key) + _KEY_BIAS
    c = u >> KEY_INDEX_BITS
    return ((1 << 63) - 1 if c == INF_COST else c), u & ((1 << KEY_INDEX_BITS) - 1)


def shard(nstarts: int, rank: int, world: int):
    """Contiguous share [lo, hi) of the starts for `rank`."""
    base, extra = divmod(nstarts, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def reduce_best(local_cost: int, local_start: int, device=None, group=None):
    """All-reduce MIN of the packed key; returns (cost, global start, owner rank
    found by the caller from the start index)."""
    import torch
    import torch.distributed as dist
    key = torch.tensor([pack_key(local_cost, local_start)], dtype=torch.int64, device=device)
    dist.all_reduce(key, op=dist.ReduceOp.MIN, group=group)
    return unpack_key(int(key.item()))


def broadcast_solution(gM, gR, src: int, device=None, group=None):
    """Broadcast the winner's setup matrices from rank `src` to all ranks."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.stack([gM, gR]).astype(np.uint8)).to(device)
    dist.broadcast(t, src=src, group=group)
    out = t.cpu().numpy()
    return out[0], out[1]


def multistart(inst, seed0: int, nstarts: int, iters: int, kmax: int = 3, mode: int = 0,
               solve=None, device=None, group=None):
    """Sharded multi-start over the ranks of the default process group.

    `solve(inst, seed0, count, iters, kmax, mode)` runs `count` starts with
    seeds seed0 .. seed0 + count - 1 and returns (best cost, best local start,
    gM, gR); by default the CUDA engine (Solver.multistart).  Returns
    (best cost, best global start, gM, gR) on every rank."""
    if not 1 <= nstarts < (1 << KEY_INDEX_BITS):
        raise ValueError(f"nstarts must be in 1 .. {(1 << KEY_INDEX_BITS) - 1}")
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    lo, hi = shard(nstarts, rank, world)
    if solve is None:
        solve = _solve_cuda
    if hi > lo:
        cost, local, gM, gR = solve(inst, seed0 + lo, hi - lo, iters, kmax, mode)
        start = lo + local
    else:
        cost, start = INF_COST, (1 << KEY_INDEX_BITS) - 1
        gM = np.zeros((inst.K, inst.T), np.uint8)
        gR = np.zeros((inst.K, inst.T), np.uint8)
    best_cost, best_start = reduce_best(cost, start, device, group)
    owner = next(r for r in range(world) if shard(nstarts, r, world)[0] <= best_start
                 < shard(nstarts, r, world)[1])
    gM, gR = broadcast_solution(gM, gR, owner, device, group)
    return best_cost, best_start, gM, gR


def _solve_cuda(inst, seed0, count, iters, kmax, mode):
    from .elsr import Solver
    with Solver(inst) as s:
        cost, local, _ = s.multistart(seed0, count, iters, kmax, mode)
        r = s.result(traj=False)
    return cost, local, r["gM"], r["gR"]
