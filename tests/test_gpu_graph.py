"""A batched scatter step captured into a CUDA graph: zero the requests'
accumulators, one persistent transport launch over every request with the
autotuned schedule, and a finalize per request.  After one step outside the
capture (which allocates the working buffers and tunes the request mix), the
captured graph replays exactly the uncaptured step's estimates, twice."""
import numpy as np
import pytest

import paper_2509_05047_gb300 as psc
import workloads as W

pytestmark = pytest.mark.gpu


def test_captured_batch_step_replays_the_uncaptured_step():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_05047_gb300 import build
    build.build()
    ctx = psc.psc_create(0)
    try:
        sc = W.scanner_tiny()
        s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
        m_id = psc.psc_load_materials(ctx, psc.materials_desc(W.standard_materials()).desc)
        l_id = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_tiny(sc)).desc)
        sn_id = psc.psc_load_sinogram(ctx, s_id, W.sensitivity_uniform(sc.lor_shape, seed=1), True)
        phs = [psc.psc_load_phantom(ctx, psc.phantom_desc(W.phantom_water_cylinder()).desc, m_id),
               psc.psc_load_phantom(ctx, psc.phantom_desc(
                   W.phantom_random_torso(8, (48, 48, 20), voxel=(4.0, 4.0, 4.0))).desc, m_id),
               psc.psc_load_phantom(ctx, psc.phantom_desc(
                   W.phantom_random_torso(9, (56, 56, 24), voxel=(3.5, 3.5, 3.5))).desc, m_id)]
        budgets = [2_000_000, 300_000, 1_200_001]
        accs = [psc.psc_acc_create(ctx, s_id) for _ in phs]
        outs = [torch.empty(sc.shape, dtype=torch.float64, device="cuda") for _ in phs]
        args = [psc.sim_args(60 + i, 7 * i, n, s_id, p, a, lut=l_id)
                for i, (p, a, n) in enumerate(zip(phs, accs, budgets))]
        sigma = (2.0, 2.0, 2.0)

        def step():
            sh = torch.cuda.current_stream().cuda_stream
            for a in accs:
                psc.psc_acc_zero(ctx, a, sh)
            psc.psc_simulate_batch_tuned(ctx, args, stream=sh)
            for a, o, n in zip(accs, outs, budgets):
                psc.psc_finalize(ctx, psc.finalize_args(a, sens=sn_id, sigma=sigma, scale=1.0 / n), o, sh)

        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            step()                                    # outside the capture: buffers, tuning
        torch.cuda.synchronize()
        ref = [o.clone() for o in outs]
        assert all(int((r != 0).sum()) > 0 for r in ref)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
            step()
        torch.cuda.synchronize()
        for _ in range(2):
            for o in outs:
                o.fill_(float("nan"))
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            for o, r in zip(outs, ref):
                assert torch.equal(o, r)
        del g
    finally:
        torch.cuda.synchronize()
        psc.psc_destroy(ctx)
