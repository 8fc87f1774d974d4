"""The bounds-checked debug build (libpsc_debug.so, PSC_DEBUG=1): every
indexed access on the hot path checks its index, records the first
violation and stays in bounds, and the launching call then fails with
PSC_EDEVICE.  Context creation self-tests the record with a known
violation.  Here the main paths (listmode and production transport, TOF
blur, gaps with edge assignment, a batched f16-LUT launch, smoothing with a
normalisation, finalize to host memory) run through it in a fresh process:
no check fires, and every result equals the release library's bit for bit."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_RUN = r'''
import sys
sys.path.insert(0, ".")
import numpy as np, torch
import paper_2509_05047_gb300 as psc
import workloads as W

def run(path):
    stream = torch.cuda.current_stream().cuda_stream
    ctx = psc.psc_create(0)
    out = {}
    try:
        mats = psc.psc_load_materials(ctx, psc.materials_desc(W.standard_materials()).desc)
        tiny = W.scanner_tiny()
        tiny.tof_sigma_mm = 20.0
        gaps = W.scanner_signa_gaps(gap_mode=2)
        s1 = psc.psc_load_scanner(ctx, psc.scanner_desc(tiny))
        s2 = psc.psc_load_scanner(ctx, psc.scanner_desc(gaps))
        p1 = psc.psc_load_phantom(ctx, psc.phantom_desc(W.phantom_water_cylinder()).desc, mats)
        l1 = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_tiny(tiny)).desc)
        l1h = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_tiny(tiny), psc.PSC_LUT_F16).desc)
        l2 = psc.psc_load_lut(ctx, psc.lut_desc(W.lut_signa(gaps)).desc)
        accs = [psc.psc_acc_create(ctx, s) for s in (s1, s1, s2, s1, s1)]
        n = 200_000
        cls = torch.empty(n, dtype=torch.int8, device="cuda")
        key = torch.empty(n, dtype=torch.int64, device="cuda")
        q = torch.empty(n, dtype=torch.int64, device="cuda")
        psc.psc_simulate(ctx, psc.sim_args(5, 0, n, s1, p1, accs[0], lut=l1, cls_out=cls, key_out=key, q_out=q),
                         stream=stream)
        psc.psc_simulate(ctx, psc.sim_args(6, 0, 1_000_000, s1, p1, accs[1], lut=l1), stream=stream)
        psc.psc_simulate(ctx, psc.sim_args(7, 0, 300_000, s2, p1, accs[2], lut=l2), stream=stream)
        psc.psc_simulate_batch(ctx, [psc.sim_args(8, 0, 400_000, s1, p1, accs[3], lut=l1h),
                                     psc.sim_args(9, 5, 100_000, s1, p1, accs[4], lut=0)], stream=stream)
        torch.cuda.synchronize()
        out["cls"], out["key"], out["q"] = cls.cpu().numpy(), key.cpu().numpy(), q.cpu().numpy()
        for i, a in enumerate(accs):
            sc = gaps if i == 2 else tiny
            t = torch.empty(sc.n_bins, dtype=torch.int64, device="cuda")
            psc.psc_acc_read(ctx, a, t, stream)
            torch.cuda.synchronize()
            idx = torch.nonzero(t).squeeze(1)
            out[f"acc{i}_idx"], out[f"acc{i}_val"] = idx.cpu().numpy(), t[idx].cpu().numpy()
        rng = np.random.default_rng(1)
        sens = psc.psc_load_sinogram(ctx, s1, rng.uniform(0.5, 1.5, tiny.lor_shape), True)
        norm = psc.psc_load_sinogram(ctx, s1, rng.uniform(0.5, 2.0, tiny.lor_shape), True)
        est = torch.empty(tiny.shape, dtype=torch.float64, device="cuda")
        psc.psc_finalize(ctx, psc.finalize_args(accs[1], sens=sens, norm=norm, sigma=(2.0, 1.5, 2.5), scale=1e-6),
                         est, stream)
        host = psc.host_tensor(tiny.shape, torch.float64)
        work = torch.empty_like(est)
        psc.psc_finalize_host(ctx, psc.finalize_args(accs[0], sens=sens, scale=1e-3), work, host, stream, stream)
        torch.cuda.synchronize()
        out["est"] = est.cpu().numpy().ravel()[::97]
        out["host"] = host.numpy().ravel()[::89].copy()
    finally:
        psc.psc_destroy(ctx)
    np.savez(path, **out)

run(sys.argv[1])
print("__OK__")
'''


def _child(env_extra, path, root):
    env = dict(os.environ)
    env.pop("PSC_LIBRARY", None)
    env.update(env_extra)
    return subprocess.run([sys.executable, "-c", _RUN, path], cwd=root, env=env, text=True,
                          capture_output=True, timeout=900)


def test_debug_build_runs_clean_and_equals_release(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_05047_gb300 import build
    build.build()
    assert os.path.exists(build.LIB_DEBUG)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    dbg, rel = str(tmp_path / "debug.npz"), str(tmp_path / "release.npz")
    r = _child({"PSC_LIBRARY": "debug"}, dbg, root)
    assert r.returncode == 0 and "__OK__" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
    r = _child({}, rel, root)
    assert r.returncode == 0 and "__OK__" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
    a, b = np.load(dbg), np.load(rel)
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert a["acc1_val"].sum() > 0 and a["acc2_val"].sum() > 0 and np.count_nonzero(a["est"]) > 0
