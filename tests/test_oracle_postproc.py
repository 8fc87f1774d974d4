"""Oracle pins for sinogram post-processing: mashing (Sec. 4), averaging
over the rotational symmetries (Sec. 2.2.4) and the smoothing-normalisation
sinogram (Sec. 2.3.2)."""
import numpy as np
import pytest

import oracle
from oracle import sinogram as S
import workloads as W


def small(n_crystals=36, n_rings=3, n_tof=5, n_rad=29):
    return W.scanner_small(n_crystals=n_crystals, n_rings=n_rings, n_tof=n_tof, n_rad=n_rad)


def test_mashing_sums_blocks_and_conserves_counts():
    rng = np.random.default_rng(1)
    x = rng.integers(0, 100, size=small().shape).astype(np.float64)
    np.testing.assert_array_equal(S.mash(x), x)
    m = S.mash(x, 3, 5)
    assert m.shape == (9, 6, 29, 1)
    np.testing.assert_array_equal(m[:, 1, :, 0], x[:, 3:6, :, :].sum(axis=(1, 3)))
    assert m.sum() == x.sum()
    with pytest.raises(ValueError):
        S.mash(x, 4, 1)


def test_rotational_average_is_a_group_average():
    """Counts are conserved (each rotation permutes the kept bins) and the
    average of an average is itself."""
    sc = small()
    x = np.random.default_rng(2).uniform(size=sc.shape)
    y = S.rotational_average(x, sc.n_crystals, sc.n_rings, 6)
    assert abs(y.sum() - x.sum()) < 1e-9 * x.sum()
    np.testing.assert_allclose(S.rotational_average(y, sc.n_crystals, sc.n_rings, 6), y, rtol=1e-12)
    with pytest.raises(ValueError):
        S.rotational_average(x, sc.n_crystals, sc.n_rings, 7)


@pytest.mark.parametrize("ca,cb,ra,rb,delta", [(0, 7, 0, 2, 31.0), (5, 30, 2, 1, -55.0), (17, 25, 1, 1, 10.0), (2, 34, 0, 1, 15.0)])
def test_rotational_average_spreads_a_bin_over_its_orbit(ca, cb, ra, rb, delta):
    """A unit count in one bin is spread evenly over the bins of the rotated
    LORs, found here with the C oracle's binning of each rotated crystal
    pair (the order reverses -> rings swap, the TOF coordinate flips; the
    deltas avoid TOF bin edges, where a flipped coordinate changes bin)."""
    sc = small()
    n, step = sc.n_crystals, 6
    st, p0, v0, r0, t0, k0 = oracle.bin_lor(sc, ca, cb, ra, rb, delta)
    assert k0 >= 0
    x = np.zeros(sc.n_bins)
    x[k0] = 1.0
    y = S.rotational_average(x.reshape(sc.shape), n, sc.n_rings, step).ravel()
    expect = np.zeros(sc.n_bins)
    for k in range(n // step):
        a, b = (ca + k * step) % n, (cb + k * step) % n
        key = oracle.bin_lor(sc, a, b, ra, rb, delta)[5] if a < b else oracle.bin_lor(sc, b, a, rb, ra, -delta)[5]
        expect[key] += 1.0 / (n // step)
    np.testing.assert_allclose(y, expect, atol=1e-15)


def test_normalisation_sinogram_of_a_constant_is_one_and_scale_free():
    sc = small()
    one = S.norm_from_sinogram(np.full(sc.shape, 7.0), sc.n_rings, (3.0, 3.0, 1.0))
    np.testing.assert_allclose(one, 1.0, rtol=1e-12)
    x = np.random.default_rng(3).uniform(0.5, 2.0, size=sc.shape)
    x[0, 0, 0, 0] = 0.0
    n1 = S.norm_from_sinogram(x, sc.n_rings, (2.0, 1.5, 1.0))
    np.testing.assert_allclose(S.norm_from_sinogram(5.0 * x, sc.n_rings, (2.0, 1.5, 1.0)), n1, rtol=1e-12)
    assert n1[0, 0, 0, 0] == 0.0
    # dividing the heavily smoothed sinogram by the normalisation restores the original
    sm = S.smooth(x, sc.n_rings, (2.0, 1.5, 1.0))
    ok = x != 0
    np.testing.assert_allclose(sm[ok] / n1[ok], x[ok], rtol=1e-12)
