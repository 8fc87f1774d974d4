"""Splitting one scatter simulation across processes (one per GPU).

Histories are independent and the random streams are counter-based, so a
request of n histories splits into contiguous history ranges, one per rank,
and every rank simulates its range into its own int64 accumulator.

The exchange is one reduction by owner.  The sinogram's ring-difference
segments (rb - ra, the planes that the axial smoothing runs along) are split
into contiguous ranges of about equal size, one per rank.  Each plane, a
contiguous [view][rad][tof] block, is summed over the ranks onto the rank
that owns its segment; runs of consecutive planes with one owner go in one
call.  Integer sums are exact and order-free, so an owned plane ends up
equal to the single-process accumulator's.  Smoothing never crosses a
segment (Sec. 2.3.2 smooths axially within a ring difference), so each rank
then finalizes its own segments alone (psc_finalize_args.seg_lo / seg_hi),
and the ranks' parts together are the single-process estimate bit for bit.

The accumulator is the caller's device tensor (psc_acc_wrap), reduced in
place: no rank holds a second accumulator-sized buffer, and each rank
finalizes 1/N of the sinogram.  NCCL reduces device tensors directly; with
gloo (CPU ranks, or tests of several processes on one GPU) each run of planes
is staged through host memory.
"""
from __future__ import annotations


def shard_range(n_histories: int, first: int, rank: int, world: int):
    """(first, count) of rank's contiguous share of [first, first + n)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(int(n_histories), int(world))
    lo = first + rank * base + min(rank, extra)
    return lo, base + (1 if rank < extra else 0)


def segment_planes(n_rings: int, seg: int) -> int:
    """Planes of ring-difference segment seg (ring difference seg - n + 1)."""
    return n_rings - abs(seg - (n_rings - 1))


def owned_segments(n_rings: int, rank: int, world: int):
    """[lo, hi) of the segments rank owns: contiguous ranges in segment order,
    a segment going to the rank whose share of the n^2 planes holds the
    segment's first plane (some ranks own none when world > 2 n - 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    total = n_rings * n_rings
    bounds, done = [], 0
    for s in range(2 * n_rings - 1):
        bounds.append(min(world - 1, done * world // total))
        done += segment_planes(n_rings, s)
    segs = [s for s, r in enumerate(bounds) if r == rank]
    return (segs[0], segs[-1] + 1) if segs else (0, 0)


def segment_of_plane(n_rings: int, plane: int) -> int:
    ra, rb = divmod(int(plane), n_rings)
    return rb - ra + n_rings - 1


def owner_runs(n_rings: int, world: int):
    """(first plane, planes, owner) runs of consecutive planes with one owner,
    covering every plane once."""
    owner = [0] * (2 * n_rings - 1)
    for r in range(world):
        lo, hi = owned_segments(n_rings, r, world)
        for s in range(lo, hi):
            owner[s] = r
    runs = []
    for p in range(n_rings * n_rings):
        o = owner[segment_of_plane(n_rings, p)]
        if runs and runs[-1][2] == o and runs[-1][0] + runs[-1][1] == p:
            runs[-1][1] += 1
        else:
            runs.append([p, 1, o])
    return [tuple(r) for r in runs]


def reduce_to_owners(acc_tensor, n_rings: int, group=None):
    """Sum the int64 accumulator (planes x bins-per-plane, any device) over
    the ranks onto each plane's owner, in place.  Planes a rank does not own
    are left with unspecified contents.  Returns this rank's (seg_lo, seg_hi)."""
    import torch
    import torch.distributed as dist
    if acc_tensor.dtype != torch.int64:
        raise TypeError("the fixed-point accumulator is int64")
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    planes = acc_tensor.view(n_rings * n_rings, -1)
    staged = acc_tensor.is_cuda and dist.get_backend(group) == "gloo"
    for p0, n, owner in owner_runs(n_rings, world):
        part = planes[p0:p0 + n]
        dst = dist.get_global_rank(group, owner) if group is not None else owner
        if staged:
            host = part.cpu()
            dist.reduce(host, dst=dst, op=dist.ReduceOp.SUM, group=group)
            if owner == rank:
                part.copy_(host)
        else:
            dist.reduce(part, dst=dst, op=dist.ReduceOp.SUM, group=group)
    return owned_segments(n_rings, rank, world)


def simulate_sharded(ctx, args, acc_tensor, n_rings: int, stream=None, group=None):
    """Run this rank's share of ``args`` (a psc SimArgs for the whole request
    whose ``acc`` wraps ``acc_tensor``, see psc_acc_wrap) and reduce the
    accumulator onto the segment owners.  Returns this rank's (first, count)
    and (seg_lo, seg_hi): finalize with ``finalize_args(..., segments=...)``."""
    import torch
    import torch.distributed as dist
    import paper_2509_05047_gb300 as psc
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    lo, cnt = shard_range(args.n_histories, args.first_history, rank, world)
    mine = psc.SimArgs.from_buffer_copy(args)
    mine.first_history, mine.n_histories = lo, cnt
    psc.psc_simulate(ctx, mine, stream=stream)
    torch.cuda.synchronize()
    segs = reduce_to_owners(acc_tensor, n_rings, group)
    torch.cuda.synchronize()
    return (lo, cnt), segs
