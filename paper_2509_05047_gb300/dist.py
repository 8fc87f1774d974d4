"""Splitting one scatter simulation across processes (one per GPU).

Histories are independent and the random streams are counter-based, so a
request of n histories splits into contiguous history ranges, one per rank;
every rank simulates its range into its own int64 accumulator, and one
integer sum over the ranks gives exactly the accumulator a single process
would have produced (integer addition is exact and order-free).  The sum is
the only exchange step; finalize then runs on the summed accumulator.
"""
from __future__ import annotations


def shard_range(n_histories: int, first: int, rank: int, world: int):
    """(first, count) of rank's contiguous share of [first, first + n)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(int(n_histories), int(world))
    lo = first + rank * base + min(rank, extra)
    return lo, base + (1 if rank < extra else 0)


def allreduce_accumulator(acc_tensor, group=None):
    """Sum an int64 accumulator tensor over all ranks in place (NCCL on GPU
    tensors, gloo on CPU tensors)."""
    import torch
    import torch.distributed as dist
    if acc_tensor.dtype != torch.int64:
        raise TypeError("the fixed-point accumulator is int64")
    dist.all_reduce(acc_tensor, op=dist.ReduceOp.SUM, group=group)
    return acc_tensor


def simulate_sharded(ctx, args, acc_id, n_bins, stream=None, group=None):
    """Run this rank's share of ``args`` (a psc SimArgs for the whole
    request) and leave the summed accumulator in ``acc_id`` on every rank.
    Returns this rank's (first, count)."""
    import torch
    import torch.distributed as dist
    import paper_2509_05047_gb300 as psc
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    lo, cnt = shard_range(args.n_histories, args.first_history, rank, world)
    mine = psc.SimArgs.from_buffer_copy(args)
    mine.first_history, mine.n_histories = lo, cnt
    psc.psc_simulate(ctx, mine, stream=stream)
    acc = torch.empty(n_bins, dtype=torch.int64, device="cuda")
    psc.psc_acc_read(ctx, acc_id, acc, stream)
    torch.cuda.synchronize()
    allreduce_accumulator(acc, group)
    psc.psc_acc_write(ctx, acc_id, acc, stream)
    torch.cuda.synchronize()
    return lo, cnt
