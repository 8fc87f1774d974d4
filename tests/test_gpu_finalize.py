"""GPU parity of the sinogram post-processing (sensitivity multiply and
normalised separable smoothing) against the oracle, from synthetic
accumulators written through the C ABI."""
import math

import numpy as np
import pytest

import oracle
import paper_2509_05047_gb300 as psc
import workloads as W

pytestmark = pytest.mark.gpu

# FP32 smoothing: three passes of <= 2K+1 positive-weight FMA sums plus the
# int64 -> FP32 conversion; each stays within ~(2K+2) * 2^-24 relative, so
# 2e-5 bounds the whole chain for K <= 32 with margin.
SMOOTH_RTOL = 2e-5


class Fin:
    def __init__(self, sc):
        import torch
        from paper_2509_05047_gb300 import build
        build.build()
        self.torch = torch
        self.sc = sc
        self.ctx = psc.psc_create(0)
        self.s_id = psc.psc_load_scanner(self.ctx, psc.scanner_desc(sc))
        self.a_id = psc.psc_acc_create(self.ctx, self.s_id)

    def write_acc(self, acc_np):
        t = self.torch.from_numpy(np.ascontiguousarray(acc_np.ravel())).cuda()
        psc.psc_acc_write(self.ctx, self.a_id, t, self.torch.cuda.current_stream().cuda_stream)
        self.torch.cuda.synchronize()

    def sino(self, host, per_lor):
        return psc.psc_load_sinogram(self.ctx, self.s_id, host, per_lor)

    def run(self, **kw):
        out = self.torch.full(self.sc.shape, np.nan, dtype=self.torch.float64, device="cuda")
        psc.psc_finalize(self.ctx, psc.finalize_args(self.a_id, **kw), out,
                         self.torch.cuda.current_stream().cuda_stream)
        self.torch.cuda.synchronize()
        return out

    def close(self):
        psc.psc_destroy(self.ctx)


@pytest.fixture(scope="module")
def small():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # ragged sizes: 38 crystals (33 radial bins kept), 9 rings, 5 TOF bins
    sc = W.scanner_small(n_crystals=38, n_rings=9, n_tof=5, n_rad=33)
    f = Fin(sc)
    rng = np.random.default_rng(0)
    f.acc = rng.integers(0, 1 << 40, size=sc.shape, dtype=np.int64)
    f.acc[rng.uniform(size=sc.shape) < 0.3] = 0
    f.write_acc(f.acc)
    f.sens_lor = rng.uniform(0.5, 1.5, size=sc.lor_shape)
    f.sens_full = rng.uniform(0.5, 1.5, size=sc.shape)
    f.norm_lor = rng.uniform(0.2, 2.0, size=sc.lor_shape)
    f.norm_lor[0, 0, :3] = 0.0
    f.ids = {k: f.sino(v, v.ndim == 3) for k, v in
             [("sens_lor", f.sens_lor), ("sens_full", f.sens_full), ("norm_lor", f.norm_lor)]}
    yield f
    f.close()


@pytest.mark.parametrize("sens", [None, "sens_lor", "sens_full"])
@pytest.mark.parametrize("scale", [1.0, 0.37])
def test_sensitivity_multiply_is_bit_exact(small, sens, scale):
    out = small.run(sens=small.ids[sens] if sens else 0, scale=scale).cpu().numpy()
    exp = oracle.finalize(small.acc, small.sc.n_rings,
                          sens=getattr(small, sens) if sens else None, scale=scale)
    np.testing.assert_array_equal(out, exp)


# the last two: the paper's chosen FWHM [9, 6, 10.5] bins, and the widths
# 4.25 / 2.12 / 7.64 of its upper bound (Sec. 2.3.2), whose axial radius
# ceil(4 x 7.64) = 31 exceeds the largest instantiated window (24) and takes
# the per-tap path, on segments shorter than the kernel
@pytest.mark.parametrize("sigma", [(2.0, 2.0, 2.0), (0.7, 3.3, 1.2), (0.0, 1.0, 0.0),
                                   (9.0 / 2.3548, 6.0 / 2.3548, 10.5 / 2.3548), (4.25, 2.12, 7.64)])
@pytest.mark.parametrize("with_norm", [False, True])
@pytest.mark.parametrize("sens_first", [False, True])
def test_smoothing_matches_oracle(small, sigma, with_norm, sens_first):
    kw = dict(sens=small.ids["sens_lor"], sigma=sigma, scale=2.5, sens_first=sens_first)
    if with_norm:
        kw["norm"] = small.ids["norm_lor"]
    out = small.run(**kw).cpu().numpy()
    exp = oracle.finalize(small.acc, small.sc.n_rings, sens=small.sens_lor,
                          norm=small.norm_lor if with_norm else None, sigma=sigma, scale=2.5,
                          smooth_before_sensitivity=not sens_first)
    assert np.all(np.isfinite(out))
    np.testing.assert_allclose(out, exp, rtol=SMOOTH_RTOL, atol=1e-300)


@pytest.mark.parametrize("with_norm", [False, True])
def test_smoothed_epilogue_is_an_exact_fp64_product(small, with_norm):
    """The smoothed path's last step is FP64: with zero-width kernels the
    FP32 passes carry y = fl32(fl32(acc) fl32(c)) [fl32(norm)] unchanged, and
    the epilogue multiplies y, widened exactly, by the FP64 reciprocal of the
    normalisation (0 where it is 0) and then by the FP64 sensitivity, each
    product rounded to nearest in FP64.  numpy's IEEE arithmetic in the same
    order gives the result bit for bit."""
    kw = dict(sens=small.ids["sens_lor"], sigma=(0.0, 0.0, 0.0), scale=2.5)
    if with_norm:
        kw["norm"] = small.ids["norm_lor"]
    out = small.run(**kw).cpu().numpy()
    y = small.acc.astype(np.float32) * np.float32(math.ldexp(2.5, -32))
    if with_norm:
        y = y * small.norm_lor.astype(np.float32)[..., None]
    x = y.astype(np.float64)
    if with_norm:
        nz = small.norm_lor != 0
        rnorm = np.where(nz, 1.0 / np.where(nz, small.norm_lor, 1.0), 0.0)
        x = x * rnorm[..., None]
    exp = x * small.sens_lor[..., None]
    np.testing.assert_array_equal(out, exp)
    # against the FP64 oracle, within the FP32 rounding of y
    ref = oracle.finalize(small.acc, small.sc.n_rings, sens=small.sens_lor,
                          norm=small.norm_lor if with_norm else None, sigma=(0.0, 0.0, 0.0), scale=2.5)
    # five FP32 roundings (acc, c, the product, norm, its product), each <= 2^-24 relative
    np.testing.assert_allclose(out, ref, rtol=6 * 2.0**-24, atol=1e-300)


@pytest.mark.parametrize("sigma", [None, (2.0, 2.0, 2.0), (4.25, 2.12, 7.64)])
@pytest.mark.parametrize("same_stream", [False, True])
def test_finalize_to_host_equals_device_finalize(small, sigma, same_stream):
    """psc_finalize_host computes the estimate in parts (plane ranges, or
    groups of ring-difference segments with smoothing) and copies each part
    to host memory as it finishes: the host copy equals psc_finalize's device
    result bit for bit, whether the copies run on their own stream or on the
    compute stream."""
    torch = small.torch
    kw = dict(sens=small.ids["sens_lor"], norm=small.ids["norm_lor"] if sigma else 0, sigma=sigma, scale=0.5)
    ref = small.run(**kw)
    host = psc.host_tensor(small.sc.shape, torch.float64)
    host.fill_(float("nan"))
    work = torch.full(small.sc.shape, np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    copy = stream if same_stream else torch.cuda.Stream()
    psc.psc_finalize_host(small.ctx, psc.finalize_args(small.a_id, **kw), work, host, stream.cuda_stream,
                          copy.cuda_stream)
    copy.synchronize()
    np.testing.assert_array_equal(host.numpy(), ref.cpu().numpy())
    torch.cuda.synchronize()
    assert torch.equal(work, ref)


@pytest.mark.parametrize("segments", [(0, 17), (3, 9), (8, 9), (16, 17)])
@pytest.mark.parametrize("sigma", [None, (2.0, 1.5, 2.0)])
def test_segment_range_finalize_to_host(small, segments, sigma):
    """A finalize restricted to ring-difference segments [lo, hi) gives, on
    those segments' planes, exactly the full finalize's values, on the
    device and copied to host memory (the copies then cover only those
    planes: rows ra (n + 1) + d of the layout)."""
    torch = small.torch
    nr = small.sc.n_rings
    kw = dict(sens=small.ids["sens_lor"], sigma=sigma, scale=1.5)
    full = small.run(**kw).cpu().numpy()
    lo, hi = segments
    planes = [ra * nr + rb for ra in range(nr) for rb in range(nr) if lo <= rb - ra + nr - 1 < hi]
    dev = small.run(segments=segments, **kw).cpu().numpy()
    np.testing.assert_array_equal(dev[planes], full[planes])
    host = psc.host_tensor(small.sc.shape, torch.float64)
    host.fill_(float("nan"))
    work = torch.empty(small.sc.shape, dtype=torch.float64, device="cuda")
    copy = torch.cuda.Stream()
    stream = torch.cuda.current_stream()
    psc.psc_finalize_host(small.ctx, psc.finalize_args(small.a_id, segments=segments, **kw), work, host,
                          stream.cuda_stream, copy.cuda_stream)
    copy.synchronize()
    h = host.numpy()
    np.testing.assert_array_equal(h[planes], full[planes])
    others = np.setdiff1d(np.arange(small.sc.n_planes), planes)
    assert np.isnan(h[others]).all()          # nothing else is copied
    with pytest.raises(psc.PscError) as e:
        small.run(segments=(5, 40), **kw)
    assert e.value.code == psc.PSC_EINVAL


def test_smoothing_conserves_mass_and_delta(small):
    acc = np.zeros(small.sc.shape, np.int64)
    acc[40, 7, 16, 2] = 1 << 32
    small.write_acc(acc)
    out = small.run(sigma=(2.0, 1.5, 1.0)).cpu().numpy()
    small.write_acc(small.acc)
    assert abs(out.sum() - 1.0) < 1e-6
    exp = oracle.finalize(acc, small.sc.n_rings, sigma=(2.0, 1.5, 1.0))
    np.testing.assert_allclose(out, exp, rtol=SMOOTH_RTOL, atol=1e-12)
    assert np.all(out[..., [0, 1, 3, 4]] == 0)


def test_smoothing_of_unaligned_accumulator(small):
    """A caller-owned accumulator 8 bytes off a 16-byte boundary (through the
    allocation-free entry point) gives the oracle's result."""
    torch = small.torch
    sc = small.sc
    store = torch.zeros(small.acc.size + 2, dtype=torch.int64, device="cuda")
    store[1:1 + small.acc.size] = torch.from_numpy(small.acc.ravel()).cuda()
    acc_t = store[1:1 + small.acc.size]
    assert acc_t.data_ptr() % 16 == 8
    sens_t = torch.from_numpy(small.sens_lor.ravel()).cuda()
    out = torch.full(sc.shape, np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    psc.psc_finalize_static(acc_t, sc.n_rings, sc.n_crystals, sc.n_rad, sc.n_tof, out, sens=sens_t,
                            sigma=(2.0, 1.5, 1.0), scale=0.5, stream=stream)
    exp = oracle.finalize(small.acc, sc.n_rings, sens=small.sens_lor, sigma=(2.0, 1.5, 1.0), scale=0.5)
    np.testing.assert_allclose(out.cpu().numpy(), exp, rtol=SMOOTH_RTOL, atol=1e-300)


def test_finalize_argument_errors(small):
    with pytest.raises(psc.PscError) as e:
        small.run(sigma=(100.0, 1.0, 1.0))
    assert e.value.code == psc.PSC_EINVAL
    with pytest.raises(psc.PscError) as e:
        small.run(sens=999)
    assert e.value.code == psc.PSC_ENOTFOUND
    other = psc.psc_load_scanner(small.ctx, psc.scanner_desc(W.scanner_small(n_crystals=16)))
    sid = psc.psc_load_sinogram(small.ctx, other, np.ones(W.scanner_small(n_crystals=16).lor_shape), True)
    with pytest.raises(psc.PscError) as e:
        small.run(sens=sid)
    assert e.value.code == psc.PSC_EINVAL


def test_paper_scale_sampled(tmp_path):
    """Full paper-scale sinogram (2025 x 224 x 447 x 27): sparse synthetic
    accumulator, sigma = 2 bins, per-LOR sensitivity and normalisation;
    sampled output bins against the brute-force oracle sum."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_signa()
    f = Fin(sc)
    try:
        idx, val = W.sparse_accumulator(sc.n_bins, 20_000_000, seed=5)
        acc = torch.zeros(sc.n_bins, dtype=torch.int64, device="cuda")
        acc[torch.from_numpy(idx).cuda()] = torch.from_numpy(val).cuda()
        psc.psc_acc_write(f.ctx, f.a_id, acc, torch.cuda.current_stream().cuda_stream)
        del acc
        sens = W.sensitivity_uniform(sc.lor_shape, seed=1)
        norm = W.sensitivity_uniform(sc.lor_shape, seed=2, lo=0.8, hi=1.2)
        s_id, n_id = f.sino(sens, True), f.sino(norm, True)

        def acc_at(flat):
            pos = np.searchsorted(idx, flat)
            pos = np.minimum(pos, idx.size - 1)
            return np.where(idx[pos] == flat, val[pos], 0)

        lor = lambda a: (lambda flat: a.ravel()[flat // sc.n_tof])
        rng = np.random.default_rng(9)
        bins = np.concatenate([rng.choice(idx, 1500), rng.integers(0, sc.n_bins, 500)])
        out = f.run(sens=s_id, norm=n_id, sigma=(2.0, 2.0, 2.0), scale=1e-3)
        got = out.view(-1)[torch.from_numpy(bins).cuda()].cpu().numpy()
        del out
        exp = oracle.finalize_at(bins, sc.shape, sc.n_rings, acc_at, lor(sens), lor(norm),
                                 (2.0, 2.0, 2.0), 1e-3)
        np.testing.assert_allclose(got, exp, rtol=SMOOTH_RTOL, atol=1e-300)
        out = f.run(sens=s_id, scale=1e-3)
        got = out.view(-1)[torch.from_numpy(bins).cuda()].cpu().numpy()
        del out
        exp = oracle.finalize_at(bins, sc.shape, sc.n_rings, acc_at, lor(sens), None, None, 1e-3)
        np.testing.assert_array_equal(got, exp)
    finally:
        f.close()


def test_fp64_products_round_like_ieee(small):
    """The FP64 multiply runs on the integer pipes: crafted operands whose
    exact products sit on rounding ties (27-bit mantissas) and accumulators
    above 2^53 must give the IEEE round-to-nearest-even result bit for bit."""
    rng = np.random.default_rng(11)
    shape = small.sc.shape
    n = int(np.prod(shape))
    acc = (rng.integers(1 << 26, 1 << 27, size=n) | 1) << rng.integers(0, 30, size=n)
    big = rng.uniform(size=n) < 0.3
    acc[big] = (1 << 53) + rng.integers(0, 1 << 20, size=big.sum())
    acc[rng.uniform(size=n) < 0.05] = 0
    acc = acc.astype(np.int64).reshape(shape)
    sens = (((rng.integers(1 << 26, 1 << 27, size=small.sc.lor_shape) | 1).astype(np.float64))
            * 2.0**-27)
    s_id = small.sino(sens, True)
    small.write_acc(acc)
    for scale in (1.0, 0.37, 3.0 * 2.0**-20):
        out = small.run(sens=s_id, scale=scale).cpu().numpy()
        np.testing.assert_array_equal(out, oracle.finalize(acc, small.sc.n_rings, sens=sens, scale=scale))
    small.write_acc(small.acc)


def test_smoothed_epilogue_rounds_ties_like_ieee(small):
    """The smoothed path's FP64 product of the FP32 value y and the FP64
    sensitivity, on operands whose exact products sit on rounding ties: with
    zero-width kernels and scale 2^32 the FP32 passes carry y = acc exactly
    (acc < 2^24), and y (24-bit odd significand) times a sensitivity with an
    odd 30-bit significand is an odd 54-bit integer times a power of two,
    halfway between two FP64 values.  Random exponents put the product's
    leading bit on both sides of the significand boundary, and plain random
    operands are mixed in; numpy's IEEE product is the expected value."""
    rng = np.random.default_rng(23)
    sc = small.sc
    s_m = rng.integers((1 << 29) + 1, 1 << 30, size=sc.lor_shape) | 1
    sens = s_m.astype(np.float64) * np.exp2(rng.integers(-20, 21, size=sc.lor_shape) - 30.0)
    lo = np.maximum(1 << 23, -(-(1 << 53) // s_m))               # y s_m >= 2^53
    hi = np.minimum((1 << 24) - 1, ((1 << 54) - 1) // s_m)        # y s_m < 2^54
    assert bool((lo <= hi).all())
    t = sc.n_tof
    y = rng.integers(lo[..., None].repeat(t, -1), hi[..., None].repeat(t, -1) + 1) | 1
    y = np.minimum(y, hi[..., None]) | 1
    y = np.where(y > hi[..., None], y - 2, y)
    plain = rng.uniform(size=sc.shape) < 0.25
    y[plain] = rng.integers(1, 1 << 24, size=int(plain.sum()))
    acc = y.astype(np.int64)
    prod = (acc.astype(object) * s_m[..., None].astype(object))[~plain]
    assert all(54 <= int(p).bit_length() <= 55 for p in prod[:1000])
    small.write_acc(acc)
    s_id = small.sino(sens, True)
    out = small.run(sens=s_id, sigma=(0.0, 0.0, 0.0), scale=2.0**32).cpu().numpy()
    np.testing.assert_array_equal(out, acc.astype(np.float64) * sens[..., None])
    small.write_acc(small.acc)


@pytest.mark.parametrize("sigma", [(2.0, 2.0, 2.0), (1.0, 0.7, 2.9), (0.6, 1.1, 0.4), (1.5, 1.0, 0.0)])
@pytest.mark.parametrize("norm_kind", [None, "lor", "bin"])
@pytest.mark.parametrize("sens_kind", ["lor", "bin"])
def test_tma_staged_axial_pass_equals_direct_pass(sigma, norm_kind, sens_kind, monkeypatch):
    """Planes whose bin count is a multiple of 4 (here 20 views x 33 radial x
    5 TOF = 3300, so the last 256-bin tile of a plane is partial) take the
    axial pass with TMA-staged shared-memory tiles; PSC_AXIAL_TMA=0 selects
    the pass that loads its rows directly.  Both must give the same bits (the
    same arithmetic per bin), for axial radii 8, 12, 2 and 0, with and without
    a normalisation, per-LOR and per-bin factors, for a segment-restricted
    call, and for the normalisation sinogram (smooth(acc) / acc); the estimate
    matches the oracle."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_small(n_crystals=40, n_rings=9, n_tof=5, n_rad=33)
    assert (sc.n_crystals // 2 * sc.n_rad * sc.n_tof) % 4 == 0
    f = Fin(sc)
    try:
        rng = np.random.default_rng(31)
        acc = rng.integers(0, 1 << 40, size=sc.shape, dtype=np.int64)
        acc[rng.uniform(size=sc.shape) < 0.3] = 0
        f.write_acc(acc)
        shp = {"lor": sc.lor_shape, "bin": sc.shape}
        sens = rng.uniform(0.5, 1.5, size=shp[sens_kind])
        norm = rng.uniform(0.2, 2.0, size=shp[norm_kind]) if norm_kind else None
        if norm is not None:
            norm.reshape(-1)[:5] = 0.0
        kw = dict(sens=f.sino(sens, sens_kind == "lor"), sigma=sigma, scale=0.37)
        if norm is not None:
            kw["norm"] = f.sino(norm, norm_kind == "lor")
        stream = torch.cuda.current_stream().cuda_stream

        def both(run):
            res = []
            for tma in ("1", "0"):
                monkeypatch.setenv("PSC_AXIAL_TMA", tma)
                out = torch.full(sc.shape, np.nan, dtype=torch.float64, device="cuda")
                run(out)
                torch.cuda.synchronize()
                res.append(out.cpu().numpy())
            np.testing.assert_array_equal(res[0], res[1])
            return res[0]

        est = both(lambda out: psc.psc_finalize(f.ctx, psc.finalize_args(f.a_id, **kw), out, stream))
        ref = oracle.finalize(acc, sc.n_rings, sens=sens, norm=norm, sigma=sigma, scale=0.37)
        np.testing.assert_allclose(est, ref, rtol=SMOOTH_RTOL, atol=1e-300)
        # segments 3 .. 11 of 17 only: their planes equal the full estimate's
        part = both(lambda out: psc.psc_finalize(f.ctx, psc.finalize_args(f.a_id, segments=(3, 12), **kw), out,
                                                 stream))
        planes = [ra * (sc.n_rings + 1) + (s - sc.n_rings + 1) + k * (sc.n_rings + 1)
                  for s in range(3, 12) for ra in [max(0, sc.n_rings - 1 - s)]
                  for k in range(sc.n_rings - abs(s - sc.n_rings + 1))]
        np.testing.assert_array_equal(part[planes], est[planes])
        if norm_kind is None and sens_kind == "lor":
            both(lambda out: psc.psc_norm_sinogram(f.ctx, f.a_id, sigma, out, stream))
    finally:
        f.close()


def test_tma_tile_wait_timeout_is_reported_and_context_stays_usable(monkeypatch):
    """The TMA-staged axial pass bounds every wait for its tile copies.  With
    PSC_FAULT_TMA_WAIT=1 each CTA first waits on an extra barrier that no copy
    completes (its real copies complete normally): the wait runs out after
    2^12 polls, the pass stops and sets the context's status word, and the
    next finalize call reports PSC_EDEVICE.  The one after it runs normally and
    gives the estimate bit for bit, so the context stays usable."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_small(n_crystals=40, n_rings=9, n_tof=5, n_rad=33)
    f = Fin(sc)
    try:
        rng = np.random.default_rng(7)
        acc = rng.integers(0, 1 << 40, size=sc.shape, dtype=np.int64)
        f.write_acc(acc)
        kw = dict(sens=f.sino(rng.uniform(0.5, 1.5, size=sc.lor_shape), True), sigma=(2.0, 2.0, 2.0), scale=0.37)
        ref = f.run(**kw).cpu().numpy()
        monkeypatch.setenv("PSC_FAULT_TMA_WAIT", "1")
        f.run(**kw)                          # enqueued normally; its waits run out on the device
        monkeypatch.delenv("PSC_FAULT_TMA_WAIT")
        with pytest.raises(psc.PscError) as e:
            f.run(**kw)
        assert e.value.code == psc.PSC_EDEVICE and "did not complete" in str(e.value)
        np.testing.assert_array_equal(f.run(**kw).cpu().numpy(), ref)
    finally:
        f.close()


@pytest.mark.parametrize("norm_kind", [None, "lor"])
def test_tma_axial_pass_on_long_segments_equals_direct_pass(norm_kind, monkeypatch):
    """With more than 36 rings the longest ring-difference segments (here 37
    to 40 planes) take the TMA-staged axial pass on 128-bin tiles in CTAs of
    128 threads, the shorter ones 256-bin tiles.  Both must give the bits of
    the pass that loads its rows directly (PSC_AXIAL_TMA=0), with and without a
    normalisation and for the normalisation sinogram; the estimate matches
    the oracle."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_small(n_crystals=40, n_rings=40, n_tof=5, n_rad=33)
    f = Fin(sc)
    try:
        rng = np.random.default_rng(41)
        acc = rng.integers(0, 1 << 40, size=sc.shape, dtype=np.int64)
        acc[rng.uniform(size=sc.shape) < 0.3] = 0
        f.write_acc(acc)
        sens = rng.uniform(0.5, 1.5, size=sc.lor_shape)
        norm = rng.uniform(0.2, 2.0, size=sc.lor_shape) if norm_kind else None
        kw = dict(sens=f.sino(sens, True), sigma=(1.5, 1.0, 2.0), scale=0.37)
        if norm is not None:
            kw["norm"] = f.sino(norm, True)
        stream = torch.cuda.current_stream().cuda_stream

        def both(run):
            res = []
            for tma in ("1", "0"):
                monkeypatch.setenv("PSC_AXIAL_TMA", tma)
                out = torch.full(sc.shape, np.nan, dtype=torch.float64, device="cuda")
                run(out)
                torch.cuda.synchronize()
                res.append(out.cpu().numpy())
            np.testing.assert_array_equal(res[0], res[1])
            return res[0]

        est = both(lambda out: psc.psc_finalize(f.ctx, psc.finalize_args(f.a_id, **kw), out, stream))
        ref = oracle.finalize(acc, sc.n_rings, sens=sens, norm=norm, sigma=(1.5, 1.0, 2.0), scale=0.37)
        np.testing.assert_allclose(est, ref, rtol=SMOOTH_RTOL, atol=1e-300)
        if norm is None:
            both(lambda out: psc.psc_norm_sinogram(f.ctx, f.a_id, (1.5, 1.0, 2.0), out, stream))
    finally:
        f.close()


def _f32_rne(v):
    """float32 nearest (ties to even) of the non-negative integer v, from its
    bits: the value the conversion must give."""
    v = int(v)
    if v < (1 << 24):
        return float(v)
    e = v.bit_length() - 24
    q, r = divmod(v, 1 << e)
    half = 1 << (e - 1)
    if r > half or (r == half and q & 1):
        q += 1
    return float(q << e)


def test_accumulator_conversion_rounds_like_ieee(small):
    """The radial pass converts int64 accumulators to FP32 on the integer
    pipes (leading bit, shift, round half to even on the dropped bits): with
    zero-width windows and scale 2^32 the estimate is that FP32 value
    widened, so every bin must equal the round-to-nearest-even FP32 value of
    its accumulator: values on rounding ties (25 significant bits, last one
    set) at every shift, ties broken only by a bit far below, values just
    under powers of two, up to 2^63 - 1, and random magnitudes."""
    rng = np.random.default_rng(17)
    shape = small.sc.shape
    n = int(np.prod(shape))
    sh = rng.integers(0, 39, size=n)
    acc = ((rng.integers(1 << 24, 1 << 25, size=n) | 1) << sh)
    sticky = rng.uniform(size=n) < 0.2
    acc[sticky] |= 1                                  # a tie broken far below
    mag = rng.uniform(size=n) < 0.3
    acc[mag] = rng.integers(0, 1 << 62, size=mag.sum()) >> rng.integers(0, 62, size=mag.sum())
    acc[:64] = [(1 << k) - 1 for k in range(1, 64)] + [0]
    acc[64:128] = [(1 << 24) + 1 + (1 << 40) * k for k in range(64)]
    acc[-1] = (1 << 63) - 1
    acc = acc.astype(np.int64).reshape(shape)
    exp = np.array([_f32_rne(v) for v in acc.ravel()]).reshape(shape)
    np.testing.assert_array_equal(exp, acc.astype(np.float32).astype(np.float64))  # numpy agrees
    small.write_acc(acc)
    np.testing.assert_array_equal(small.run(sigma=(0.0, 0.0, 0.0), scale=2.0**32).cpu().numpy(), exp)
    small.write_acc(small.acc)
