"""Oracle pins: sensitivity multiply and normalised Gaussian smoothing."""
import math

import numpy as np
import pytest

import oracle
from oracle import sinogram as F


def _brute_force_smooth(x, n_rings, sigma):
    """Direct 3D product-kernel sum, loop over every output bin (tiny grids)."""
    g1, g2, g3 = (F.gaussian_weights(s) for s in sigma)
    K1, K2, K3 = g1.size // 2, g2.size // 2, g3.size // 2
    P, V, Rr, T = x.shape
    out = np.zeros_like(x)
    segs = F.segment_planes(n_rings)
    where = {}
    for s in segs:
        for j, p in enumerate(s):
            where[int(p)] = (s, j)
    for p in range(P):
        seg, j = where[p]
        for v in range(V):
            for r in range(Rr):
                acc = np.zeros(T)
                for a in range(-K3, K3 + 1):
                    pp = seg[F.reflect_index(j + a, len(seg))]
                    for b in range(-K2, K2 + 1):
                        vv = F.reflect_index(v + b, V)
                        for c in range(-K1, K1 + 1):
                            rr = F.reflect_index(r + c, Rr)
                            acc += g3[a + K3] * g2[b + K2] * g1[c + K1] * x[pp, vv, rr]
                out[p, v, r] = acc
    return out


def test_gaussian_weights_and_reflection():
    g = F.gaussian_weights(2.0)
    assert g.size == 17 and abs(g.sum() - 1) < 1e-15
    np.testing.assert_allclose(g, g[::-1], rtol=0, atol=0)
    k = np.arange(-8, 9)
    np.testing.assert_allclose(g / g[8], np.exp(-k**2 / 8.0), rtol=1e-14)
    np.testing.assert_array_equal(F.reflect_index([-3, -2, -1, 0, 4, 5, 6, 7], 5), [2, 1, 0, 0, 4, 4, 3, 2])
    np.testing.assert_array_equal(F.reflect_index([-1, -2, 1, 2, 3], 1), [0, 0, 0, 0, 0])


def test_segments_partition_planes():
    for n in (1, 2, 5, 16):
        segs = F.segment_planes(n)
        allp = np.sort(np.concatenate(segs))
        np.testing.assert_array_equal(allp, np.arange(n * n))
        for s in segs:
            ra, rb = s // n, s % n
            assert np.all(np.diff(ra) == 1) and len(set(rb - ra)) == 1


def test_separable_equals_brute_force_3d():
    rng = np.random.default_rng(0)
    n_rings = 3
    x = rng.uniform(size=(9, 5, 7, 2))
    sig = (1.1, 0.7, 0.9)
    np.testing.assert_allclose(F.smooth(x, n_rings, sig), _brute_force_smooth(x, n_rings, sig),
                               rtol=1e-12, atol=1e-14)


def test_delta_response_is_normalised_kernel():
    n_rings, V, Rr, T = 5, 30, 41, 3
    x = np.zeros((n_rings * n_rings, V, Rr, T))
    # plane (ra=2, rb=2): the centre of the 5-plane direct segment
    p = 2 * n_rings + 2
    x[p, 15, 20, 1] = 1.0
    sig = (2.0, 1.5, 0.8)
    y = F.smooth(x, n_rings, sig)
    g1, g2, g3 = (F.gaussian_weights(s) for s in sig)
    K1, K2, K3 = g1.size // 2, g2.size // 2, g3.size // 2
    seg = [ra * n_rings + ra for ra in range(n_rings)]
    expect = np.zeros_like(x)
    for a in range(-K3, K3 + 1):
        pp = seg[int(F.reflect_index(2 + a, 5))]
        expect[pp, 15 - K2:15 + K2 + 1, 20 - K1:20 + K1 + 1, 1] += g3[a + K3] * np.outer(g2, g1)
    np.testing.assert_allclose(y, expect, atol=1e-16)
    assert abs(y.sum() - 1.0) < 1e-14
    assert np.all(y[:, :, :, [0, 2]] == 0)            # TOF bins are not mixed


def test_mass_is_conserved_with_reflection():
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(16, 6, 9, 2))
    y = F.smooth(x, 4, (3.0, 2.5, 2.0))               # kernels wider than some axes
    np.testing.assert_allclose(y.sum(axis=(0, 1, 2)), x.sum(axis=(0, 1, 2)), rtol=1e-12)


def test_sensitivity_multiply_is_elementwise():
    rng = np.random.default_rng(2)
    acc = rng.integers(0, 1 << 45, size=(4, 3, 5, 2), dtype=np.int64)
    sens = rng.uniform(0.5, 1.5, size=(4, 3, 5))
    out = F.finalize(acc, 2, sens=sens, scale=0.25)
    np.testing.assert_array_equal(out, (acc.astype(np.float64) * 2.0**-34) * sens[..., None])
    full = rng.uniform(0.5, 1.5, size=acc.shape)
    np.testing.assert_array_equal(F.finalize(acc, 2, sens=full), acc * 2.0**-32 * full)


def test_normalised_smoothing_order():
    """x * norm -> smooth -> / norm -> * sens (Sec. 2.3.2); a constant
    normalisation cancels; zero normalisation bins give zero."""
    rng = np.random.default_rng(3)
    acc = rng.integers(0, 1 << 40, size=(9, 4, 6, 2), dtype=np.int64)
    sens = rng.uniform(0.5, 1.5, size=(9, 4, 6))
    sig = (1.0, 1.0, 1.0)
    plain = F.finalize(acc, 3, sens=sens, sigma=sig)
    const = F.finalize(acc, 3, sens=sens, norm=np.full((9, 4, 6), 3.0), sigma=sig)
    np.testing.assert_allclose(plain, const, rtol=1e-13)
    norm = rng.uniform(0.5, 2.0, size=(9, 4, 6))
    norm[0, 0, 0] = 0.0
    y = F.finalize(acc, 3, sens=sens, norm=norm, sigma=sig)
    x = acc * 2.0**-32
    expect = F.smooth(x * norm[..., None], 3, sig) / np.where(norm == 0, 1, norm)[..., None] * sens[..., None]
    expect[0, 0, 0] = 0.0
    np.testing.assert_allclose(y, expect, rtol=1e-13)
    y2 = F.finalize(acc, 3, sens=sens, sigma=sig, smooth_before_sensitivity=False)
    np.testing.assert_allclose(y2, F.smooth(x * sens[..., None], 3, sig), rtol=1e-13)


@pytest.mark.parametrize("order", [True, False])
def test_sampled_finalize_equals_full(order):
    rng = np.random.default_rng(4)
    shape = (16, 10, 13, 3)
    acc = rng.integers(0, 1 << 40, size=shape, dtype=np.int64)
    sens = rng.uniform(0.5, 1.5, size=shape[:3])
    norm = rng.uniform(0.5, 1.5, size=shape[:3])
    sig = (1.3, 0.9, 1.1)
    full = F.finalize(acc, 4, sens=sens, norm=norm, sigma=sig, scale=3.0,
                      smooth_before_sensitivity=order)
    bins = rng.choice(acc.size, 300, replace=False)
    lor = lambda a: (lambda flat: a.ravel()[flat // shape[3]])
    got = F.finalize_at(bins, shape, 4, lambda flat: acc.ravel()[flat], lor(sens), lor(norm),
                        sig, 3.0, order)
    np.testing.assert_allclose(got, full.ravel()[bins], rtol=1e-12)
