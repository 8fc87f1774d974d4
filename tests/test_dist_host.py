"""Multi-rank host logic on the CPU (gloo, world size 2): a request split by
history ranges, each plane summed onto the rank that owns its ring-difference
segment, equals the single-process accumulator on the owned planes bit for
bit, and each rank's finalize of its own segments equals the single-process
estimate there (smoothing never crosses a segment)."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2509_05047_gb300.dist import (owned_segments, owner_runs, segment_of_plane,
                                         segment_planes, shard_range)


def test_shards_partition_the_range():
    for n, first, world in [(10, 0, 3), (1_000_003, 17, 8), (5, 2**40, 8), (0, 0, 2)]:
        spans = [shard_range(n, first, r, world) for r in range(world)]
        assert sum(c for _, c in spans) == n
        pos = first
        for lo, c in spans:
            assert lo == pos
            pos += c
        assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 0, 2, 2)


@pytest.mark.parametrize("n_rings,world", [(1, 1), (4, 2), (4, 4), (9, 3), (45, 8), (45, 2), (3, 8)])
def test_segment_owners_partition_the_sinogram(n_rings, world):
    n_seg = 2 * n_rings - 1
    spans = [owned_segments(n_rings, r, world) for r in range(world)]
    owned = [s for lo, hi in spans for s in range(lo, hi)]
    assert owned == list(range(n_seg))                      # every segment once, in rank order
    planes = [sum(segment_planes(n_rings, s) for s in range(lo, hi)) for lo, hi in spans]
    assert sum(planes) == n_rings * n_rings
    if world <= n_seg:
        assert max(planes) <= n_rings * n_rings / world + n_rings
    covered = []
    for p0, n, owner in owner_runs(n_rings, world):
        for p in range(p0, p0 + n):
            lo, hi = spans[owner]
            assert lo <= segment_of_plane(n_rings, p) < hi
            covered.append(p)
    assert covered == list(range(n_rings * n_rings))


def _scanner_phantom():
    import workloads as W
    return (W.scanner_small(n_crystals=32, n_rings=4, n_tof=5, radius=200.0),
            W.phantom_water_cylinder(dims=(24, 24, 8), voxel=(4.0, 4.0, 4.0), radius=40.0))


def _rank(rank, world, port, n, out_path):
    import torch
    import torch.distributed as dist
    import oracle
    import workloads as W
    from paper_2509_05047_gb300.dist import reduce_to_owners
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc, ph = _scanner_phantom()
    lo, cnt = shard_range(n, 5, rank, world)
    r = oracle.simulate(sc, W.standard_materials(), ph, None, 99, lo, cnt, threads=2, acc=True)
    acc = torch.from_numpy(r["acc"].ravel().copy())
    segs = reduce_to_owners(acc, sc.n_rings)
    np.save(out_path % rank, acc.numpy())
    np.save((out_path % rank) + ".segs.npy", np.array(segs))
    dist.destroy_process_group()


def test_reduce_to_owners_equals_single_process(tmp_path):
    import oracle
    import workloads as W
    n, world = 60_001, 2
    out = str(tmp_path / "acc%d.npy")
    port = 29500 + (os.getpid() % 1000)
    mp.spawn(_rank, args=(world, port, n, out), nprocs=world, join=True)
    sc, ph = _scanner_phantom()
    ref = oracle.simulate(sc, W.standard_materials(), ph, None, 99, 5, n, threads=2, acc=True)["acc"]
    sens = W.sensitivity_uniform(sc.lor_shape, seed=2)
    full = oracle.finalize(ref, sc.n_rings, sens=sens, sigma=(2.0, 1.5, 2.0), scale=1e-3)
    seen = []
    for rank in range(world):
        got = np.load(out % rank).reshape(sc.shape)
        lo, hi = np.load((out % rank) + ".segs.npy")
        planes = [p for p in range(sc.n_planes) if lo <= segment_of_plane(sc.n_rings, p) < hi]
        seen += planes
        assert got[planes].sum() > 0
        np.testing.assert_array_equal(got[planes], ref[planes])
        # the rank's finalize of its own segments: planes it does not own hold
        # partial sums, and smoothing within segments never reads them
        part = oracle.finalize(got, sc.n_rings, sens=sens, sigma=(2.0, 1.5, 2.0), scale=1e-3)
        np.testing.assert_array_equal(part[planes], full[planes])
    assert sorted(seen) == list(range(sc.n_planes))
