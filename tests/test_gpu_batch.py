"""Batched launches: several requests (different phantoms, scanners, LUT
precisions and history budgets) in one persistent launch give each request
exactly the accumulator and listmode it gets alone."""
import numpy as np
import pytest

import paper_2509_05047_gb300 as psc
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_05047_gb300 import build
    build.build()
    c = psc.psc_create(0)
    yield c
    psc.psc_destroy(c)


def _acc(ctx, a_id, n_bins):
    import torch
    t = torch.empty(n_bins, dtype=torch.int64, device="cuda")
    psc.psc_acc_read(ctx, a_id, t, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_batch_equals_each_request_alone(ctx):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    mats = psc.psc_load_materials(ctx, psc.materials_desc(W.standard_materials()).desc)
    tiny = W.scanner_tiny()
    small = W.scanner_small(n_crystals=64, n_rings=8, n_tof=7, radius=200.0, ring_pitch=6.0,
                            tof_bin_mm=30.0, tof_sigma_mm=20.0, e_lo=350.0)
    s1 = psc.psc_load_scanner(ctx, psc.scanner_desc(tiny))
    s2 = psc.psc_load_scanner(ctx, psc.scanner_desc(small))
    p1 = psc.psc_load_phantom(ctx, psc.phantom_desc(W.phantom_water_cylinder()).desc, mats)
    p2 = psc.psc_load_phantom(ctx, psc.phantom_desc(
        W.phantom_random_torso(3, (40, 40, 16), voxel=(4.0, 4.0, 4.0))).desc, mats)
    p3 = psc.psc_load_phantom(ctx, psc.phantom_desc(
        W.phantom_random_torso(4, (48, 48, 20), voxel=(3.0, 3.0, 3.0))).desc, mats)
    l1 = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_tiny(tiny)).desc)
    l2 = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_tiny(tiny), psc.PSC_LUT_F16).desc)
    l3 = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_smooth(8, 6, 6, small.module_t, small.module_a,
                                                          small.e_lo)).desc)
    jobs = [  # (scanner, phantom, lut, seed, first, n)
        (s1, p1, l1, 11, 0, 150_001), (s1, p2, l2, 12, 7, 20_000), (s2, p3, l3, 13, 1_000, 333),
        (s2, p3, 0, 14, 5, 90_000), (s1, p1, 0, 15, 0, 1)]
    scanners = {s1: tiny, s2: small}
    accs = [psc.psc_acc_create(ctx, sc) for sc, *_ in jobs]
    alone, lm_alone = [], []
    for (sc, ph, lu, seed, first, n), a in zip(jobs, accs):
        cls = torch.empty(n, dtype=torch.int8, device="cuda")
        key = torch.empty(n, dtype=torch.int64, device="cuda")
        psc.psc_simulate(ctx, psc.sim_args(seed, first, n, sc, ph, a, lut=lu, cls_out=cls, key_out=key),
                         stream=stream)
        alone.append(_acc(ctx, a, scanners[sc].n_bins))
        lm_alone.append((cls.cpu().numpy(), key.cpu().numpy()))
        psc.psc_acc_zero(ctx, a, stream)
    lms = [(torch.empty(n, dtype=torch.int8, device="cuda"), torch.empty(n, dtype=torch.int64, device="cuda"))
           for *_, n in jobs]
    batch = [psc.sim_args(seed, first, n, sc, ph, a, lut=lu, cls_out=c, key_out=k)
             for (sc, ph, lu, seed, first, n), a, (c, k) in zip(jobs, accs, lms)]
    st = psc.psc_simulate_batch(ctx, batch, stats=True, stream=stream)
    assert sum(st[c] for c in psc.CLASSES) == sum(j[-1] for j in jobs)
    for i, ((sc, *_), a) in enumerate(zip(jobs, accs)):
        np.testing.assert_array_equal(_acc(ctx, a, scanners[sc].n_bins), alone[i])
        np.testing.assert_array_equal(lms[i][0].cpu().numpy(), lm_alone[i][0])
        np.testing.assert_array_equal(lms[i][1].cpu().numpy(), lm_alone[i][1])
    assert sum(int(x.sum() > 0) for x in alone) >= 3


def test_batch_of_many_jobs_equals_one_range(ctx):
    """60 jobs (more than one launch holds) covering consecutive history
    ranges of one stream add up to the single request over the union."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    sc = W.scanner_tiny()
    mats = psc.psc_load_materials(ctx, psc.materials_desc(W.standard_materials()).desc)
    s = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
    p = psc.psc_load_phantom(ctx, psc.phantom_desc(W.phantom_water_cylinder()).desc, mats)
    a1, a2 = psc.psc_acc_create(ctx, s), psc.psc_acc_create(ctx, s)
    edges = np.unique(np.concatenate([[0, 400_000], np.random.default_rng(1).integers(0, 400_000, 59)]))
    batch = [psc.sim_args(21, int(lo), int(hi - lo), s, p, a1) for lo, hi in zip(edges[:-1], edges[1:])]
    assert len(batch) > 48
    psc.psc_simulate_batch(ctx, batch, stream=stream)
    psc.psc_simulate(ctx, psc.sim_args(21, 0, 400_000, s, p, a2), stream=stream)
    np.testing.assert_array_equal(_acc(ctx, a1, sc.n_bins), _acc(ctx, a2, sc.n_bins))


def test_tuned_batch_equals_untuned_batch(ctx):
    """The autotuned batched launch (probes of candidate schedules on slices
    of every request's own histories, then the fastest on the rest) gives
    every request exactly the accumulator of the default schedule; a second
    call on the same request mix takes the cached choice without probes."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    mats = psc.psc_load_materials(ctx, psc.materials_desc(W.standard_materials()).desc)
    tiny = W.scanner_tiny()
    s1 = psc.psc_load_scanner(ctx, psc.scanner_desc(tiny))
    l1 = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_tiny(tiny)).desc)
    phs = [psc.psc_load_phantom(ctx, psc.phantom_desc(W.phantom_water_cylinder()).desc, mats),
           psc.psc_load_phantom(ctx, psc.phantom_desc(
               W.phantom_random_torso(5, (48, 48, 20), voxel=(4.0, 4.0, 4.0))).desc, mats),
           psc.psc_load_phantom(ctx, psc.phantom_desc(
               W.phantom_random_torso(6, (64, 64, 24), voxel=(3.5, 3.5, 3.5))).desc, mats)]
    budgets = [3_000_001, 250_000, 1_700_000]
    acc_u = [psc.psc_acc_create(ctx, s1) for _ in phs]
    acc_t = [psc.psc_acc_create(ctx, s1) for _ in phs]

    def args(accs, seed0):
        return [psc.sim_args(seed0 + i, 13 * i, n, s1, p, a, lut=l1)
                for i, (p, a, n) in enumerate(zip(phs, accs, budgets))]

    psc.psc_simulate_batch(ctx, args(acc_u, 40), stream=stream)
    first = psc.psc_simulate_batch_tuned(ctx, args(acc_t, 40), stream=stream)
    assert first["probed"] >= 4 and first["rate"] > 0 and first["block"] in (256, 512)
    for a, b in zip(acc_u, acc_t):
        u = _acc(ctx, a, tiny.n_bins)
        assert u.sum() > 0
        np.testing.assert_array_equal(_acc(ctx, b, tiny.n_bins), u)
    for a in acc_t:
        psc.psc_acc_zero(ctx, a, stream)
    again = psc.psc_simulate_batch_tuned(ctx, args(acc_t, 40), stream=stream)
    assert again["probed"] == 0 and again["block"] == first["block"]
    for a, b in zip(acc_u, acc_t):
        np.testing.assert_array_equal(_acc(ctx, b, tiny.n_bins), _acc(ctx, a, tiny.n_bins))
    with pytest.raises(psc.PscError):
        key = torch.empty(10, dtype=torch.int64, device="cuda")
        psc.psc_simulate_batch_tuned(ctx, [psc.sim_args(1, 0, 10, s1, phs[0], acc_t[0], key_out=key)],
                                     stream=stream)
