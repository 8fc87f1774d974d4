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


def _sparse(keys, qs):
    """Sorted (bin, summed weight) pairs of a list of binned events."""
    u, inv = np.unique(keys, return_inverse=True)
    v = np.zeros(u.size, np.int64)
    np.add.at(v, inv, qs)
    return u, v


def _check_against_oracle(sc, r, g_idx, g_val, est_at, n, sigma, i):
    """The GPU's iteration i (its accumulator's non-zero bins g_idx, g_val and
    its estimate est_at(bins)) against the oracle run r of the same range."""
    import oracle
    K = int(np.ceil(4 * max(sigma[0], sigma[1])))
    shape = sc.shape
    m = r["cls"] == oracle.SCATTER
    o_idx, o_val = _sparse(r["key"][m], r["q"][m])
    # bins whose sums differ beyond the weight tolerance: mismatched histories
    allb = np.union1d(o_idx, g_idx)
    ov = np.zeros(allb.size, np.int64)
    gv = np.zeros(allb.size, np.int64)
    ov[np.searchsorted(allb, o_idx)] = o_val
    gv[np.searchsorted(allb, g_idx)] = g_val
    bad = allb[np.abs(gv - ov) > 1e-5 * np.maximum(ov, gv) + 1]
    assert bad.size <= 2 + 0.002 * m.sum(), (bad.size, m.sum())
    # sampled bins: every event bin, neighbours and random bins, away from the
    # bad bins' smoothing neighbourhood (same TOF bin and segment, views and
    # radial bins within the kernel radius)
    srng = np.random.default_rng(i)
    cand = np.concatenate([allb, allb + shape[3], allb - shape[3] * shape[2],
                           srng.integers(0, sc.n_bins, 20_000)])
    cand = np.unique(cand[(cand >= 0) & (cand < sc.n_bins)])

    def coords(b):
        t = b % shape[3]
        rr = (b // shape[3]) % shape[2]
        v = (b // (shape[3] * shape[2])) % shape[1]
        p = b // (shape[3] * shape[2] * shape[1])
        return p % sc.n_rings - p // sc.n_rings, v, rr, t

    cd, cv, cr, ct = coords(cand)
    ok = np.ones(cand.size, bool)
    for b in bad:
        bd, bv, br, bt = coords(np.array([b]))
        ok &= ~((cd == bd) & (ct == bt) & (np.abs(cv - bv) <= K) & (np.abs(cr - br) <= K))
    sample = cand[ok]
    assert sample.size > 10_000

    def acc_at(flat):
        j = np.clip(np.searchsorted(o_idx, flat), 0, o_idx.size - 1)
        return np.where(o_idx[j] == flat, o_val[j], 0)

    exp = np.concatenate([oracle.finalize_at(sample[k:k + 1500], shape, sc.n_rings, acc_at,
                                             sigma=sigma, scale=1.0 / n)
                          for k in range(0, sample.size, 1500)])
    val = est_at(sample)
    assert np.count_nonzero(exp) > 2_000
    # FP32 smoothing (2e-5) of weights within 1e-5 of the oracle's
    np.testing.assert_allclose(val, exp, rtol=3e-5, atol=1e-12 * exp.max())


def test_joint_iterations_match_the_oracle():
    """Each iteration of the joint loop (Sec. 2.3.3: a new activity image,
    a short simulation, smoothing) against the oracle: the oracle simulates
    the same activity and history range, and its FP64 smoothing formula
    (oracle.finalize_at) gives the expected estimate at every bin that a
    scatter event of either side reaches and at random bins, away from the
    few bins where a mismatched history (< 0.1 %) lands."""
    import torch
    import oracle
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_tiny()
    mats, ph, lut = W.standard_materials(), W.phantom_water_cylinder(), W.lut_tiny(sc)
    s = Session(sc, mats, ph, lut)
    sigma, n, seed, n_iter = (2.0, 2.0, 2.0), 1_000_000, 4242, 2
    try:
        stream = s.stream()
        out = torch.empty(sc.shape, dtype=torch.float64, device="cuda")
        acts = [ph.activity.astype(np.float32)]
        rng = np.random.default_rng(8)
        got = []

        def reconstruct(est, i):
            nxt = (acts[-1] * rng.uniform(0.25, 1.75, size=acts[-1].shape)).astype(np.float32)
            acts.append(nxt)
            return nxt

        def keep(i, o):
            acc = s.acc()
            idx = torch.nonzero(acc).squeeze(1)
            got.append((idx.cpu().numpy(), acc[idx].cpu().numpy(), o.clone()))

        scatter_iterations(s.ctx, s.s_id, s.p_id, s.a_id, acts[0], reconstruct, n_iter, n, seed, out,
                           lut=s.l_id, sigma=sigma, stream=stream, on_estimate=keep)
        torch.cuda.synchronize()
        for i, (g_idx, g_val, est) in enumerate(got):
            phi = W.Phantom(ph.dims, ph.voxel, ph.origin, ph.material, ph.density, acts[i])
            r = oracle.simulate(sc, mats, phi, lut, seed, i * n, n, threads=8)
            _check_against_oracle(sc, r, g_idx, g_val,
                                  lambda b: est.view(-1)[torch.from_numpy(b).cuda()].cpu().numpy(),
                                  n, sigma, i)
    finally:
        s.close()
