"""Multi-rank host logic on the CPU (gloo, world size 2): a request split by
history ranges and summed with one int64 all-reduce equals the single-process
result bit for bit."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2509_05047_gb300.dist import shard_range


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


def _rank(rank, world, port, n, out_path):
    import torch
    import torch.distributed as dist
    import oracle
    import workloads as W
    from paper_2509_05047_gb300.dist import allreduce_accumulator
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = W.scanner_small(n_crystals=32, n_rings=4, n_tof=5, radius=200.0)
    ph = W.phantom_water_cylinder(dims=(24, 24, 8), voxel=(4.0, 4.0, 4.0), radius=40.0)
    lo, cnt = shard_range(n, 5, rank, world)
    r = oracle.simulate(sc, W.standard_materials(), ph, None, 99, lo, cnt, threads=2, acc=True)
    acc = torch.from_numpy(r["acc"].ravel().copy())
    allreduce_accumulator(acc)
    if rank == 0:
        np.save(out_path, acc.numpy())
    dist.destroy_process_group()


def test_sharded_sum_equals_single_process(tmp_path):
    import oracle
    import workloads as W
    n, world = 60_001, 2
    out = str(tmp_path / "acc.npy")
    port = 29500 + (os.getpid() % 1000)
    mp.spawn(_rank, args=(world, port, n, out), nprocs=world, join=True)
    sc = W.scanner_small(n_crystals=32, n_rings=4, n_tof=5, radius=200.0)
    ph = W.phantom_water_cylinder(dims=(24, 24, 8), voxel=(4.0, 4.0, 4.0), radius=40.0)
    ref = oracle.simulate(sc, W.standard_materials(), ph, None, 99, 5, n, threads=2, acc=True)
    got = np.load(out)
    assert got.sum() > 0
    np.testing.assert_array_equal(got, ref["acc"].ravel())
