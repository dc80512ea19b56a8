"""Seed sharding over ranks: one process per GPU, each holding a replica of the graph.

The solves of different seeds are independent (each reads the graph and writes only its own
accumulators, Eq. local-gd run per source), so a batch of seeds is cut into contiguous
blocks, one per rank, and no data moves between ranks while they solve.  The only
collectives are outside the solve: a max over ranks of the step time, a sum of counters,
and an optional gather of the per-seed top-k lists onto rank 0.

Works with any torch.distributed backend (gloo on CPU tensors, NCCL on CUDA tensors): every
collective is issued on tensors of the caller's device.
"""
from __future__ import annotations


def shard_bounds(total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block [lo, hi) of `total` items owned by `rank` of `world`; block sizes
    differ by at most one and the first `total % world` ranks take the larger blocks."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError(f"bad shard request total={total} world={world} rank={rank}")
    q, r = divmod(total, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def shard_seeds(seeds, world: int, rank: int):
    """This rank's block of a global seed list (a view)."""
    lo, hi = shard_bounds(len(seeds), world, rank)
    return seeds[lo:hi]


def _dist():
    import torch.distributed as dist
    if not dist.is_initialized():
        raise RuntimeError("torch.distributed is not initialised")
    return dist


def max_over_ranks(value: float, device="cpu") -> float:
    """The maximum of a per-rank scalar (e.g. a step time) over all ranks."""
    import torch
    dist = _dist()
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device="cpu") -> float:
    """The sum of a per-rank scalar (e.g. pushed edges) over all ranks."""
    import torch
    dist = _dist()
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_topk(ids, vals, total: int):
    """Assemble the per-seed top-k lists of every rank's block on rank 0.

    ids (int32) and vals (float32) are this rank's [block, k] tensors for the block that
    shard_bounds(total, world, rank) names.  Returns the [total, k] tensors on rank 0 (in the
    global seed order) and None elsewhere.  Blocks are padded to the largest block for the
    all-gather (NCCL has no ragged gather); padding rows are dropped again on rank 0.
    """
    import torch
    dist = _dist()
    world, rank = dist.get_world_size(), dist.get_rank()
    lo, hi = shard_bounds(total, world, rank)
    if ids.shape[0] != hi - lo or vals.shape != ids.shape:
        raise ValueError(f"rank {rank}: expected [{hi - lo}, k] ids and vals, got {tuple(ids.shape)} "
                         f"and {tuple(vals.shape)}")
    k = ids.shape[1]
    width = shard_bounds(total, world, 0)[1]  # rank 0 holds a largest block
    pi = torch.full((width, k), -1, dtype=torch.int32, device=ids.device)
    pv = torch.zeros((width, k), dtype=torch.float32, device=ids.device)
    pi[: hi - lo] = ids
    pv[: hi - lo] = vals
    gi = [torch.empty_like(pi) for _ in range(world)]
    gv = [torch.empty_like(pv) for _ in range(world)]
    dist.all_gather(gi, pi)
    dist.all_gather(gv, pv)
    if rank != 0:
        return None
    rows_i, rows_v = [], []
    for r in range(world):
        a, b = shard_bounds(total, world, r)
        rows_i.append(gi[r][: b - a])
        rows_v.append(gv[r][: b - a])
    return torch.cat(rows_i), torch.cat(rows_v)

