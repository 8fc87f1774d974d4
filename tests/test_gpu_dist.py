"""One request split across two processes (world size 2, gloo through host
memory, both ranks on the one GPU: no kernel of one rank waits on the
other's).  Each rank simulates its history range into its own caller-owned
accumulator (psc_acc_wrap), the planes are summed onto the ranks that own
their ring-difference segments, and each rank finalizes its own segments;
together they equal one process running the whole request, bit for bit."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

SIGMA = (2.0, 2.0, 2.0)


def _rank(rank, world, port, n, seed, out_path):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    import paper_2509_05047_gb300 as psc
    import workloads as W
    from paper_2509_05047_gb300.dist import simulate_sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    sc = W.scanner_tiny()
    ctx = psc.psc_create(0)
    try:
        s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
        m_id = psc.psc_load_materials(ctx, psc.materials_desc(W.standard_materials()).desc)
        p_id = psc.psc_load_phantom(ctx, psc.phantom_desc(W.phantom_water_cylinder()).desc, m_id)
        l_id = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_tiny(sc)).desc)
        sn_id = psc.psc_load_sinogram(ctx, s_id, W.sensitivity_uniform(sc.lor_shape, seed=1), True)
        acc = torch.zeros(sc.n_bins, dtype=torch.int64, device="cuda")
        a_id = psc.psc_acc_wrap(ctx, s_id, acc)
        stream = torch.cuda.current_stream().cuda_stream
        args = psc.sim_args(seed, 11, n, s_id, p_id, a_id, lut=l_id)
        (lo, cnt), segs = simulate_sharded(ctx, args, acc, sc.n_rings, stream=stream)
        out = torch.full(sc.shape, float("nan"), dtype=torch.float64, device="cuda")
        psc.psc_finalize(ctx, psc.finalize_args(a_id, sens=sn_id, sigma=SIGMA, scale=1.0 / n, segments=segs),
                         out, stream)
        torch.cuda.synchronize()
        np.save(out_path % rank, out.cpu().numpy())
        np.save((out_path % rank) + ".meta.npy", np.array([lo, cnt, segs[0], segs[1]]))
    finally:
        psc.psc_destroy(ctx)
        dist.destroy_process_group()


def test_two_ranks_equal_one_process(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_05047_gb300 as psc
    import workloads as W
    from paper_2509_05047_gb300 import build
    from paper_2509_05047_gb300.dist import segment_of_plane
    build.build()
    n, seed, world = 3_000_001, 77, 2
    out = str(tmp_path / "est%d.npy")
    port = 29600 + (os.getpid() % 1000)
    mp.start_processes(_rank, args=(world, port, n, seed, out), nprocs=world, join=True, start_method="spawn")
    # one process, the whole request
    sc = W.scanner_tiny()
    ctx = psc.psc_create(0)
    try:
        s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
        m_id = psc.psc_load_materials(ctx, psc.materials_desc(W.standard_materials()).desc)
        p_id = psc.psc_load_phantom(ctx, psc.phantom_desc(W.phantom_water_cylinder()).desc, m_id)
        l_id = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_tiny(sc)).desc)
        sn_id = psc.psc_load_sinogram(ctx, s_id, W.sensitivity_uniform(sc.lor_shape, seed=1), True)
        a_id = psc.psc_acc_create(ctx, s_id)
        stream = torch.cuda.current_stream().cuda_stream
        psc.psc_simulate(ctx, psc.sim_args(seed, 11, n, s_id, p_id, a_id, lut=l_id), stream=stream)
        ref = torch.empty(sc.shape, dtype=torch.float64, device="cuda")
        psc.psc_finalize(ctx, psc.finalize_args(a_id, sens=sn_id, sigma=SIGMA, scale=1.0 / n), ref, stream)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
    finally:
        psc.psc_destroy(ctx)
    seen, total = [], 0
    for rank in range(world):
        est = np.load(out % rank)
        lo, cnt, s_lo, s_hi = np.load((out % rank) + ".meta.npy")
        total += cnt
        planes = [p for p in range(sc.n_planes) if s_lo <= segment_of_plane(sc.n_rings, p) < s_hi]
        assert planes
        seen += planes
        np.testing.assert_array_equal(est[planes], ref[planes])
    assert total == n and sorted(seen) == list(range(sc.n_planes))
    assert np.count_nonzero(ref) > 0


def test_acc_wrap_checks_its_memory():
    """psc_acc_wrap takes 8-byte-aligned device memory of the context's device
    only, and a wrapped accumulator is not freed by psc_unload."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_05047_gb300 as psc
    import workloads as W
    from paper_2509_05047_gb300 import build
    build.build()
    sc = W.scanner_small(n_crystals=16, n_rings=4, n_tof=5)
    ctx = psc.psc_create(0)
    try:
        s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
        t = torch.zeros(sc.n_bins + 1, dtype=torch.int64, device="cuda")
        before = psc.psc_resident_bytes(ctx)
        a = psc.psc_acc_wrap(ctx, s_id, t)
        assert psc.psc_resident_bytes(ctx) == before        # not counted against the budget
        t[:sc.n_bins] = 7
        out = torch.empty(sc.n_bins, dtype=torch.int64, device="cuda")
        psc.psc_acc_read(ctx, a, out, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert int(out.sum()) == 7 * sc.n_bins
        psc.psc_unload(ctx, a)
        t.fill_(1)                                          # still the caller's memory
        torch.cuda.synchronize()
        odd = t.view(torch.uint8)[4:4 + 8 * sc.n_bins]
        for bad in (odd, t.cpu(), None):
            with pytest.raises((psc.PscError, TypeError, AttributeError)) as e:
                psc.psc_acc_wrap(ctx, s_id, bad)
            if isinstance(e.value, psc.PscError):
                assert e.value.code == psc.PSC_EINVAL
    finally:
        psc.psc_destroy(ctx)
