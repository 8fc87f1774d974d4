"""GPU parity of the sinogram post-processing calls against the oracle:
mashing and the rotational-symmetry sum on int64 accumulators (bit-exact),
the smoothing-normalisation sinogram (smoothing tolerance)."""
import numpy as np
import pytest

import oracle
from oracle import sinogram as S
import paper_2509_05047_gb300 as psc
import workloads as W

pytestmark = pytest.mark.gpu

SMOOTH_RTOL = 2e-5   # the smoothing tolerance of the finalize tests


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_05047_gb300 import build
    build.build()
    ctx = psc.psc_create(0)
    yield ctx, torch
    psc.psc_destroy(ctx)


def _acc(ctx, torch, sc, values):
    s_id = psc.psc_load_scanner(ctx, psc.scanner_desc(sc))
    a_id = psc.psc_acc_create(ctx, s_id)
    t = torch.from_numpy(np.ascontiguousarray(values.ravel())).cuda()
    psc.psc_acc_write(ctx, a_id, t, torch.cuda.current_stream().cuda_stream)
    return s_id, a_id


@pytest.mark.parametrize("vf,tf", [(1, 1), (2, 1), (3, 5), (18, 1)])
def test_mashing_matches_oracle(env, vf, tf):
    ctx, torch = env
    sc = W.scanner_small(n_crystals=36, n_rings=3, n_tof=5, n_rad=29)
    x = np.random.default_rng(vf * 10 + tf).integers(0, 1 << 40, size=sc.shape, dtype=np.int64)
    _, a_id = _acc(ctx, torch, sc, x)
    out = torch.full((sc.n_planes, sc.n_views // vf, sc.n_rad, sc.n_tof // tf), -1, dtype=torch.int64, device="cuda")
    psc.psc_acc_mash(ctx, a_id, vf, tf, out, torch.cuda.current_stream().cuda_stream)
    np.testing.assert_array_equal(out.cpu().numpy(), S.mash(x, vf, tf))
    with pytest.raises(psc.PscError) as e:
        psc.psc_acc_mash(ctx, a_id, 4, 1, out)
    assert e.value.code == psc.PSC_EINVAL


# n / step even: one thread per orbit; odd: one thread per output bin
@pytest.mark.parametrize("n_crystals,n_rad,step", [(36, 29, 6), (36, 35, 4), (38, 33, 19), (36, 29, 2),
                                                   (36, 33, 18), (40, 39, 8), (40, 37, 5)])
def test_rotation_sum_matches_oracle(env, n_crystals, n_rad, step):
    ctx, torch = env
    sc = W.scanner_small(n_crystals=n_crystals, n_rings=3, n_tof=4, n_rad=n_rad)
    x = np.random.default_rng(n_crystals + step).integers(0, 1 << 40, size=sc.shape, dtype=np.int64)
    s_id, a_id = _acc(ctx, torch, sc, x)
    o_id = psc.psc_acc_create(ctx, s_id)
    stream = torch.cuda.current_stream().cuda_stream
    psc.psc_acc_rotate_sum(ctx, a_id, step, o_id, stream)
    got = torch.empty(sc.n_bins, dtype=torch.int64, device="cuda")
    psc.psc_acc_read(ctx, o_id, got, stream)
    exp = S.rotational_average(x, n_crystals, sc.n_rings, step, average=False)
    np.testing.assert_array_equal(got.cpu().numpy().reshape(sc.shape), exp)
    with pytest.raises(psc.PscError):
        psc.psc_acc_rotate_sum(ctx, a_id, step, a_id, stream)


def test_rotation_sum_on_the_paper_scanner_conserves_and_is_a_group_sum(env):
    """448 x 45 crystals, modules of 16: 28 rotations (14 views per orbit).
    The total is 28 times the input's, and summing a rotation sum again
    multiplies it by 28."""
    ctx, torch = env
    sc = W.scanner_small(n_crystals=448, n_rings=4, n_tof=3, n_rad=447)
    rng = np.random.default_rng(5)
    x = np.zeros(sc.n_bins, np.int64)
    idx = rng.integers(0, sc.n_bins, size=20_000)
    x[idx] = rng.integers(1, 1 << 30, size=idx.size)
    s_id, a_id = _acc(ctx, torch, sc, x)
    o1, o2 = psc.psc_acc_create(ctx, s_id), psc.psc_acc_create(ctx, s_id)
    stream = torch.cuda.current_stream().cuda_stream
    psc.psc_acc_rotate_sum(ctx, a_id, 16, o1, stream)
    psc.psc_acc_rotate_sum(ctx, o1, 16, o2, stream)
    r1 = torch.empty(sc.n_bins, dtype=torch.int64, device="cuda")
    r2 = torch.empty_like(r1)
    psc.psc_acc_read(ctx, o1, r1, stream)
    psc.psc_acc_read(ctx, o2, r2, stream)
    assert int(r1.sum()) == 28 * int(x.sum())
    assert bool((r2 == 28 * r1).all())
    exp = S.rotational_average(x.reshape(sc.shape), 448, sc.n_rings, 16, average=False)
    np.testing.assert_array_equal(r1.cpu().numpy().reshape(sc.shape), exp)


def test_normalisation_sinogram_matches_oracle(env):
    ctx, torch = env
    sc = W.scanner_small(n_crystals=38, n_rings=9, n_tof=5, n_rad=33)
    rng = np.random.default_rng(7)
    x = rng.integers(1 << 20, 1 << 36, size=sc.shape, dtype=np.int64)
    x[rng.uniform(size=sc.shape) < 0.2] = 0
    _, a_id = _acc(ctx, torch, sc, x)
    out = torch.full(sc.shape, np.nan, dtype=torch.float64, device="cuda")
    sigma = (4.0, 3.0, 2.0)
    psc.psc_norm_sinogram(ctx, a_id, sigma, out, torch.cuda.current_stream().cuda_stream)
    got = out.cpu().numpy()
    exp = S.norm_from_sinogram(x.astype(np.float64), sc.n_rings, sigma)
    assert np.all(got[x == 0] == 0.0)
    np.testing.assert_allclose(got, exp, rtol=SMOOTH_RTOL, atol=1e-300)


@pytest.mark.parametrize("n_rings,span", [(9, 1), (9, 3), (9, 5), (9, 7), (9, 17), (11, 3)])
def test_span_mashing_matches_oracle(env, n_rings, span):
    """Span (segment) mashing: the output plane count and every exact int64
    sum equal the oracle's brute force over the input planes."""
    ctx, torch = env
    sc = W.scanner_small(n_crystals=38, n_rings=n_rings, n_tof=3, n_rad=33)
    rng = np.random.default_rng(span * 31 + n_rings)
    acc = rng.integers(0, 1 << 40, size=sc.shape, dtype=np.int64)
    s_id, a_id = _acc(ctx, torch, sc, acc)
    exp = S.span_mash(acc, n_rings, span)
    planes = psc.psc_acc_span(ctx, a_id, span)
    assert planes == exp.shape[0]
    out = torch.full((planes,) + sc.shape[1:], -1, dtype=torch.int64, device="cuda")
    assert psc.psc_acc_span(ctx, a_id, span, out, torch.cuda.current_stream().cuda_stream) == planes
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), exp)
    with pytest.raises(psc.PscError) as e:
        psc.psc_acc_span(ctx, a_id, 2)
    assert e.value.code == psc.PSC_EINVAL
    psc.psc_unload(ctx, a_id)
    psc.psc_unload(ctx, s_id)
