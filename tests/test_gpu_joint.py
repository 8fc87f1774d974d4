"""The joint activity/scatter iteration driver (Sec. 2.4.2, third
scenario): each iteration's estimate equals a standalone simulation and
finalize of that iteration's activity and history range, the caller's
reconstruction sees every estimate in order, and the activity it returns
drives the next iteration."""
import numpy as np
import pytest

import paper_2509_05047_gb300 as psc
import workloads as W
from paper_2509_05047_gb300.joint import scatter_iterations

from gpu_helpers import Session

pytestmark = pytest.mark.gpu


def test_scatter_iterations_match_standalone_runs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_tiny()
    mats, ph, lut = W.standard_materials(), W.phantom_water_cylinder(), W.lut_tiny(sc)
    s = Session(sc, mats, ph, lut)
    try:
        n, seed, n_iter = 300_000, 99, 3
        stream = s.stream()
        out = torch.empty(sc.shape, dtype=torch.float64, device="cuda")
        seen, acts = [], [ph.activity.astype(np.float32)]
        rng = np.random.default_rng(4)

        def reconstruct(est, i):
            # a stand-in for the caller's reconstruction: it must see iteration i's estimate
            seen.append((i, float(est.sum())))
            nxt = (acts[-1] * rng.uniform(0.5, 1.5, size=acts[-1].shape)).astype(np.float32)
            acts.append(nxt)
            return nxt

        estimates = []
        last = scatter_iterations(s.ctx, s.s_id, s.p_id, s.a_id, acts[0], reconstruct, n_iter, n, seed, out,
                                  lut=s.l_id, sigma=(2.0, 2.0, 2.0), stream=stream,
                                  on_estimate=lambda i, o: estimates.append(o.clone()))
        torch.cuda.synchronize()
        assert len(estimates) == n_iter and [i for i, _ in seen] == list(range(n_iter - 1))
        assert last is acts[-1]
        for i, total in seen:
            assert total == float(estimates[i].sum())
        for i, est in enumerate(estimates):
            # the same activity and history range, run by hand
            psc.psc_update_activity(s.ctx, s.p_id, acts[i])
            s.zero()
            psc.psc_simulate(s.ctx, psc.sim_args(seed, i * n, n, s.s_id, s.p_id, s.a_id, lut=s.l_id),
                             stream=stream)
            ref = torch.empty_like(out)
            psc.psc_finalize(s.ctx, psc.finalize_args(s.a_id, sigma=(2.0, 2.0, 2.0), scale=1.0 / n), ref, stream)
            torch.cuda.synchronize()
            assert torch.equal(est, ref)
        # different activities give different estimates
        assert not torch.equal(estimates[0], estimates[1])
        with pytest.raises(ValueError):
            scatter_iterations(s.ctx, s.s_id, s.p_id, s.a_id, acts[0], reconstruct, 0, n, seed, out)
    finally:
        s.close()
