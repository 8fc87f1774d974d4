"""Oracle pins: Philox4x32-10, uniforms, Vose alias table, emission."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert list(oracle.philox4x32_10(ctr, key)) == out


def test_alias_reconstructs_distribution():
    rng = np.random.default_rng(0)
    a = rng.exponential(size=1000).astype(np.float32)
    a[rng.integers(0, 1000, 100)] = 0.0
    prob, alias = oracle.alias_build(a)
    n = a.size
    target = a.astype(np.float64) * n / a.astype(np.float64).sum()
    got = prob.copy()
    mask = alias != np.arange(n)
    np.add.at(got, alias[mask], 1.0 - prob[mask])
    np.testing.assert_allclose(got, target, rtol=0, atol=1e-9)
    assert np.all((prob >= 0) & (prob <= 1.0))
    assert np.all(prob[a == 0] == 0.0)


def test_alias_rejects_bad_activity():
    with pytest.raises(ValueError):
        oracle.alias_build(np.zeros(10, np.float32))
    with pytest.raises(ValueError):
        oracle.alias_build(np.array([1.0, -1.0], np.float32))
    with pytest.raises(ValueError):
        oracle.alias_build(np.array([1.0, np.nan], np.float32))


def _vacuum_phantom(dims, activity):
    nx, ny, nz = dims
    ph = W.phantom_uniform_box(dims=dims, voxel=(4.0, 4.0, 4.0), material=W.MAT_VACUUM,
                               density=0.0, source="uniform")
    ph.activity[:] = activity.reshape(nz, ny, nx)
    return ph


def test_emission_voxel_frequencies_match_activity():
    rng = np.random.default_rng(1)
    dims = (8, 8, 4)
    act = rng.uniform(0.0, 3.0, size=256).astype(np.float32)
    act[::7] = 0.0
    ph = _vacuum_phantom(dims, act)
    sc = W.scanner_tiny()
    n = 200_000
    r = oracle.simulate(sc, W.standard_materials(), ph, None, 99, 0, n, threads=8, records=True)
    vox = r["rec"]["voxel"]
    counts = np.bincount(vox, minlength=256)
    assert counts[act == 0].sum() == 0
    expect = act.astype(np.float64) / act.sum() * n
    m = expect > 0
    chi2 = ((counts[m] - expect[m]) ** 2 / expect[m]).sum()
    assert stats.chi2.sf(chi2, m.sum() - 1) > 0.01


def test_emission_point_in_voxel_and_isotropic():
    dims = (16, 12, 8)
    ph = _vacuum_phantom(dims, np.ones(16 * 12 * 8, np.float32))
    n = 100_000
    r = oracle.simulate(W.scanner_tiny(), W.standard_materials(), ph, None, 7, 1000, n,
                        threads=8, records=True)["rec"]
    v = r["voxel"]
    ix, iy, iz = v % 16, (v // 16) % 12, v // (16 * 12)
    lo = np.stack([ph.origin[0] + ix * 4.0, ph.origin[1] + iy * 4.0, ph.origin[2] + iz * 4.0], 1)
    assert np.all(r["emit"] >= lo) and np.all(r["emit"] < lo + 4.0)
    d = r["dir"]
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)
    # cos(theta) uniform on [-1, 1], phi uniform on [0, 2 pi)
    c_hist = np.histogram(d[:, 2], bins=20, range=(-1, 1))[0]
    p_hist = np.histogram(np.arctan2(d[:, 1], d[:, 0]), bins=20, range=(-np.pi, np.pi))[0]
    for h in (c_hist, p_hist):
        assert stats.chisquare(h).pvalue > 0.01
    # photon 2 leaves back to back: with no attenuation its exit direction is -dir
    np.testing.assert_allclose(r["exit_dir"][:, 1], -d, atol=0)
    np.testing.assert_allclose(r["exit_dir"][:, 0], d, atol=0)


def test_counter_based_streams_are_partition_independent():
    sc = W.scanner_tiny()
    mats = W.standard_materials()
    ph = W.phantom_water_cylinder()
    full = oracle.simulate(sc, mats, ph, None, 5, 100, 3000, threads=1)
    a = oracle.simulate(sc, mats, ph, None, 5, 100, 1234, threads=3)
    b = oracle.simulate(sc, mats, ph, None, 5, 1334, 1766, threads=2)
    for k in ("cls", "key", "q"):
        np.testing.assert_array_equal(full[k], np.concatenate([a[k], b[k]]))
