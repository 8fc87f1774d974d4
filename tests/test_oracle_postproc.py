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


def test_span_mashing_hand_example():
    """3 rings, span 3: ring differences -1..1 form segment 0 (axial sums
    z = 0..4), d = +-2 the outer segments (z = 2 only).  With plane p holding
    the value p (plane = ra 3 + rb): segment -1 is (2, 0) = 6; segment 0 is
    z=0: (0,0) = 0, z=1: (0,1) + (1,0) = 4, z=2: (1,1) = 4, z=3: (1,2) + (2,1)
    = 12, z=4: (2,2) = 8; segment +1 is (0, 2) = 2."""
    assert oracle.span_segments(3, 3) == [(-1, -2, -2, [2]), (0, -1, 1, [0, 1, 2, 3, 4]), (1, 2, 2, [2])]
    s = np.arange(9, dtype=np.int64).reshape(9, 1, 1, 1)
    np.testing.assert_array_equal(oracle.span_mash(s, 3, 3).ravel(), [6, 0, 4, 4, 12, 8, 2])


@pytest.mark.parametrize("n_rings,span", [(9, 1), (9, 3), (9, 5), (9, 7), (9, 17), (45, 3), (45, 11)])
def test_span_mashing_conserves_counts_and_plane_count(n_rings, span):
    rng = np.random.default_rng(n_rings * 100 + span)
    s = rng.integers(0, 1 << 30, size=(n_rings * n_rings, 2, 3, 2), dtype=np.int64)
    out = oracle.span_mash(s, n_rings, span)
    np.testing.assert_array_equal(out.sum(axis=0), s.sum(axis=0))
    segs = oracle.span_segments(n_rings, span)
    assert out.shape[0] == sum(len(zs) for *_, zs in segs)
    # every ring difference falls in exactly one segment, and every output
    # plane receives at least one input plane
    ds = [d for _, lo, hi, _ in segs for d in range(lo, hi + 1)]
    ones = oracle.span_mash(np.ones((n_rings * n_rings, 1, 1, 1), np.int64), n_rings, span).ravel()
    assert ones.min() >= 1 and ones.sum() == n_rings * n_rings
    assert sorted(ds) == list(range(-(n_rings - 1), n_rings))


def test_span_one_is_a_plane_permutation():
    n = 7
    s = (np.arange(n * n, dtype=np.int64) * 1000 + 7).reshape(n * n, 1, 1, 1)
    out = oracle.span_mash(s, n, 1).ravel()
    assert out.size == n * n and sorted(out) == sorted(s.ravel())


def test_one_segment_is_the_anti_diagonal_sums():
    """A span covering every ring difference (2 n - 1) leaves one segment whose
    plane z is the sum over ra + rb = z."""
    n = 6
    rng = np.random.default_rng(4)
    s = rng.integers(0, 100, size=(n * n, 1, 2, 1), dtype=np.int64)
    out = oracle.span_mash(s, n, 2 * n - 1)
    assert out.shape[0] == 2 * n - 1
    for z in range(2 * n - 1):
        want = sum(s[ra * n + (z - ra)] for ra in range(n) if 0 <= z - ra < n)
        np.testing.assert_array_equal(out[z], want)
