"""psc_finalize_static: the smoothed scatter estimate for callers that cannot
allocate device memory (their memory is owned by another allocator, capped,
or must not be allocated once a real-time loop runs).  It is checked against
psc_finalize, the entry point that owns its working memory, on two calls in
a row; the second call must not see the first call's leftovers.

Collected last on purpose (file name), so that a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

import paper_2509_05047_gb300 as psc
import workloads as W

pytestmark = pytest.mark.gpu

SMOOTH_RTOL = 2e-5   # the smoothing tolerance of the other finalize tests


def _static(acc_t, sc, sens_t, norm_t, sigma, scale, sens_first, out_t, stream):
    psc.psc_finalize_static(acc_t, sc.n_rings, sc.n_crystals, sc.n_rad, sc.n_tof, out_t,
                            sens=sens_t, norm=norm_t, sigma=sigma, scale=scale,
                            sens_first=sens_first, stream=stream)


def test_static_finalize_matches_allocating_finalize():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_05047_gb300 import build
    build.build()
    sc = W.scanner_small(n_crystals=38, n_rings=9, n_tof=5, n_rad=33)
    rng = np.random.default_rng(21)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    ctx = psc.psc_create(0)
    try:
        s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
        a_id = psc.psc_acc_create(ctx, s_id)
        cases = [((2.0, 2.0, 2.0), 1.0, False, True), ((0.7, 3.3, 1.2), 0.25, True, False)]
        free_after = []
        for sigma, scale, sens_first, with_norm in cases:
            acc = rng.integers(0, 1 << 40, size=sc.shape, dtype=np.int64)
            acc[rng.uniform(size=sc.shape) < 0.3] = 0
            sens = rng.uniform(0.5, 1.5, size=sc.lor_shape)
            norm = rng.uniform(0.2, 2.0, size=sc.lor_shape)
            acc_t = torch.from_numpy(acc.ravel()).to(dev)
            sens_t = torch.from_numpy(sens.ravel()).to(dev)
            norm_t = torch.from_numpy(norm.ravel()).to(dev) if with_norm else None
            # reference: the allocating entry point on the same inputs
            psc.psc_acc_write(ctx, a_id, acc_t, stream)
            sn = psc.psc_load_sinogram(ctx, s_id, sens, True)
            nn = psc.psc_load_sinogram(ctx, s_id, norm, True) if with_norm else 0
            ref = torch.empty(sc.shape, dtype=torch.float64, device=dev)
            psc.psc_finalize(ctx, psc.finalize_args(a_id, sens=sn, norm=nn, sigma=sigma, scale=scale,
                                                    sens_first=sens_first), ref, stream)
            out = torch.full(sc.shape, np.nan, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            _static(acc_t, sc, sens_t, norm_t, sigma, scale, sens_first, out, stream)
            torch.cuda.synchronize()
            free_after.append((free_before, torch.cuda.mem_get_info()[0]))
            np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=SMOOTH_RTOL,
                                       atol=1e-300)
        # after the first call (which may load the library's static array),
        # a call leaves the device's free memory unchanged
        assert free_after[1][0] == free_after[1][1]
        # sizes beyond the static working memory are rejected with a clear error
        big = W.scanner_signa()
        with pytest.raises(psc.PscError) as e:
            _static(acc_t, big, None, None, (2.0, 2.0, 2.0), 1.0, False, out, stream)
        assert e.value.code == psc.PSC_EOVERFLOW and "working memory" in str(e.value)
    finally:
        psc.psc_destroy(ctx)
