"""psc_finalize_static: the smoothed scatter estimate for callers that cannot
allocate device memory (their memory is owned by another allocator, capped,
or must not be allocated once a real-time loop runs).  It is checked against
psc_finalize, the entry point that owns its working memory, on two calls in
a row for each case; a call must not see an earlier call's leftovers.

Collected last on purpose (file name), so that a run that stops at the first
failure has already run every other test."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2509_05047_gb300 as psc
import workloads as W

pytestmark = pytest.mark.gpu

SMOOTH_RTOL = 2e-5   # the smoothing tolerance of the other finalize tests
STATIC_BYTES = 64 << 20


def _static(acc_t, sc, sens_t, norm_t, sigma, scale, sens_first, out_t, stream, sens_per_lor=True,
            norm_per_lor=True):
    psc.psc_finalize_static(acc_t, sc.n_rings, sc.n_crystals, sc.n_rad, sc.n_tof, out_t,
                            sens=sens_t, sens_per_lor=sens_per_lor, norm=norm_t,
                            norm_per_lor=norm_per_lor, sigma=sigma, scale=scale,
                            sens_first=sens_first, stream=stream)


def _require_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_05047_gb300 import build
    build.build()
    return torch


def _compare(torch, ctx, s_id, a_id, sc, rng, cases, stream):
    """Each case on fresh inputs, twice in a row through the static entry
    point, against psc_finalize on the same inputs."""
    dev = torch.device("cuda:0")
    free_after = []
    for sigma, scale, sens_first, sens_kind, norm_kind in cases:
        acc = rng.integers(0, 1 << 40, size=sc.shape, dtype=np.int64)
        acc[rng.uniform(size=sc.shape) < 0.3] = 0
        shp = {"lor": sc.lor_shape, "bin": sc.shape}
        sens = rng.uniform(0.5, 1.5, size=shp[sens_kind]) if sens_kind else None
        norm = rng.uniform(0.2, 2.0, size=shp[norm_kind]) if norm_kind else None
        if norm is not None:
            norm.reshape(-1)[:7] = 0.0          # zero normalisation values give 0
        acc_t = torch.from_numpy(acc.ravel()).to(dev)
        sens_t = torch.from_numpy(sens.ravel()).to(dev) if sens is not None else None
        norm_t = torch.from_numpy(norm.ravel()).to(dev) if norm is not None else None
        # reference: the allocating entry point on the same inputs
        psc.psc_acc_write(ctx, a_id, acc_t, stream)
        sn = psc.psc_load_sinogram(ctx, s_id, sens, sens_kind == "lor") if sens is not None else 0
        nn = psc.psc_load_sinogram(ctx, s_id, norm, norm_kind == "lor") if norm is not None else 0
        ref = torch.empty(sc.shape, dtype=torch.float64, device=dev)
        psc.psc_finalize(ctx, psc.finalize_args(a_id, sens=sn, norm=nn, sigma=sigma, scale=scale,
                                                sens_first=sens_first), ref, stream)
        for _ in range(2):
            out = torch.full(sc.shape, np.nan, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            _static(acc_t, sc, sens_t, norm_t, sigma, scale, sens_first, out, stream,
                    sens_per_lor=sens_kind != "bin", norm_per_lor=norm_kind != "bin")
            torch.cuda.synchronize()
            free_after.append((free_before, torch.cuda.mem_get_info()[0]))
            if sigma is None:
                assert torch.equal(out, ref)     # the exact FP64 multiply
            else:
                np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=SMOOTH_RTOL,
                                           atol=1e-300)
            del out
        for i in (sn, nn):
            if i:
                psc.psc_unload(ctx, i)
        del acc_t, sens_t, norm_t, ref
    return free_after


def test_static_finalize_matches_allocating_finalize():
    torch = _require_gpu()
    sc = W.scanner_small(n_crystals=38, n_rings=9, n_tof=5, n_rad=33)
    rng = np.random.default_rng(21)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = psc.psc_create(0)
    try:
        s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
        a_id = psc.psc_acc_create(ctx, s_id)
        cases = [((2.0, 2.0, 2.0), 1.0, False, "lor", "lor"),
                 ((0.7, 3.3, 1.2), 0.25, True, "lor", None),
                 (None, 0.5, False, "lor", None),                 # no smoothing
                 (None, 2.0, False, "bin", None),
                 (None, 1.0, False, None, None),
                 ((1.5, 1.0, 2.5), 1.0, False, "bin", "bin"),     # per-bin sensitivity and normalisation
                 ((1.5, 1.0, 2.5), 3.0, True, "bin", "lor"),
                 ((2.0, 0.5, 1.0), 1.0, False, None, "bin")]      # no sensitivity
        free_after = _compare(torch, ctx, s_id, a_id, sc, rng, cases, stream)
        # after the first smoothing call (which may map the library's static
        # array), no call changes the device's free memory
        assert all(b == a for b, a in free_after[1:]), free_after
        # sizes beyond the static working memory are rejected with a clear error
        acc_t = torch.zeros(8, dtype=torch.int64, device="cuda")
        out = torch.zeros(8, dtype=torch.float64, device="cuda")
        big = W.scanner_signa()
        with pytest.raises(psc.PscError) as e:
            _static(acc_t, big, None, None, (2.0, 2.0, 2.0), 1.0, False, out, stream)
        assert e.value.code == psc.PSC_EOVERFLOW and "working memory" in str(e.value)
        # the sinogram shapes psc_load_scanner accepts, no others
        bad = W.scanner_small(n_crystals=38, n_rings=9, n_tof=5, n_rad=33)
        bad.n_rad = 34                                             # 37 - 34 is odd
        with pytest.raises(psc.PscError) as e:
            _static(acc_t, bad, None, None, (2.0, 2.0, 2.0), 1.0, False, out, stream)
        assert e.value.code == psc.PSC_EINVAL
        with pytest.raises(psc.PscError) as e:
            psc.psc_load_scanner(ctx, psc.scanner_desc(bad))
        assert e.value.code == psc.PSC_EINVAL
    finally:
        psc.psc_destroy(ctx)


def test_static_finalize_near_its_size_limit():
    """A per-bin normalisation fills the static array most (4 + 8 bytes per
    bin): a 5.16 M-bin sinogram (92 % of 64 MiB) gives the allocating entry
    point's result; one TOF bin more exceeds the array and is rejected, and
    the same sinogram with a per-LOR normalisation (4 bytes per bin + 8 per
    LOR) fits."""
    torch = _require_gpu()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(5)
    ctx = psc.psc_create(0)
    try:
        sc = W.scanner_small(n_crystals=64, n_rings=16, n_tof=10, n_rad=63)
        assert 0.9 * STATIC_BYTES < 12 * sc.n_bins + 256 <= STATIC_BYTES
        s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
        a_id = psc.psc_acc_create(ctx, s_id)
        _compare(torch, ctx, s_id, a_id, sc, rng, [((1.0, 2.0, 1.5), 1.0, False, "lor", "bin")], stream)
        sc11 = W.scanner_small(n_crystals=64, n_rings=16, n_tof=11, n_rad=63)
        acc_t = torch.zeros(sc11.n_bins, dtype=torch.int64, device="cuda")
        norm_t = torch.ones(sc11.n_bins, dtype=torch.float64, device="cuda")
        out = torch.empty(sc11.n_bins, dtype=torch.float64, device="cuda")
        with pytest.raises(psc.PscError) as e:
            _static(acc_t, sc11, None, norm_t, (1.0, 1.0, 1.0), 1.0, False, out, stream, norm_per_lor=False)
        assert e.value.code == psc.PSC_EOVERFLOW
        _static(acc_t, sc11, None, norm_t[:sc11.n_bins // sc11.n_tof], (1.0, 1.0, 1.0), 1.0, False, out,
                stream)
        torch.cuda.synchronize()
        assert bool((out == 0).all())
    finally:
        psc.psc_destroy(ctx)


_FIRST_CALL = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, ".")
import paper_2509_05047_gb300 as psc
import workloads as W
sc = W.scanner_small(n_crystals=38, n_rings=9, n_tof=5, n_rad=33)
acc = torch.from_numpy(np.random.default_rng(1).integers(0, 1 << 40, sc.n_bins)).cuda()
outs = [torch.empty(sc.n_bins, dtype=torch.float64, device="cuda") for _ in range(2)]
s = torch.cuda.current_stream().cuda_stream
free = []
for o in outs:
    torch.cuda.synchronize()
    f0 = torch.cuda.mem_get_info()[0]
    psc.psc_finalize_static(acc, sc.n_rings, sc.n_crystals, sc.n_rad, sc.n_tof, o, sigma=(2.0, 2.0, 2.0), stream=s)
    torch.cuda.synchronize()
    free.append((f0, torch.cuda.mem_get_info()[0]))
print(json.dumps({"free": free, "same": bool(torch.equal(outs[0], outs[1]))}))
'''


def test_first_call_in_a_fresh_process_maps_only_the_static_array():
    """In a process whose first use of the library is this entry point, the
    first smoothing call may map the static array (lazy module loading): it
    takes at most 64 MiB plus the allocation granularity and the module's
    code; the second call takes nothing, and both give the same result."""
    torch = _require_gpu()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    env.pop("CUDA_MODULE_LOADING", None)
    out = subprocess.check_output([sys.executable, "-c", _FIRST_CALL], cwd=root, env=env, text=True,
                                  timeout=600)
    r = json.loads(out.strip().splitlines()[-1])
    (b0, a0), (b1, a1) = r["free"]
    assert r["same"]
    assert 0 <= b0 - a0 <= STATIC_BYTES + (8 << 20), (b0 - a0)
    assert b1 == a1
