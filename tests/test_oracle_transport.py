"""Oracle pins: Woodcock tracking against exact attenuation, vacuum geometry,
invariants, symmetry and Poisson statistics of the sinogram."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads as W


def _mu511(mats, phantom):
    """Linear attenuation (mm^-1) of every voxel at 511 keV (table node 511)."""
    tot = np.array([m.compton[511] + m.rayleigh[511] + m.photo[511] for m in mats])
    return phantom.density.astype(np.float64) * tot[phantom.material] / 10.0


def _box_exit(p, d, lo, hi):
    """Distance along d from p (inside) to the boundary of the box [lo, hi)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(d > 0, (hi - p) / d, np.where(d < 0, (lo - p) / d, np.inf))
    return t.min(axis=1)


def _optical_depth(p, d, mu, phantom, h=0.5, seed=0):
    """Unbiased line integral of mu from p along d to the grid boundary by
    randomly offset midpoint sampling (independent of the oracle)."""
    rng = np.random.default_rng(seed)
    lo = np.array(phantom.origin)
    vox = np.array(phantom.voxel)
    dims = np.array(phantom.dims)
    hi = lo + dims * vox
    L = _box_exit(p, d, lo, hi)
    tau = np.zeros(p.shape[0])
    nmax = int(np.ceil(L.max() / h)) + 1
    for s in range(0, p.shape[0], 4000):
        pp, dd, LL = p[s:s + 4000], d[s:s + 4000], L[s:s + 4000]
        u = rng.uniform(size=(pp.shape[0], 1))
        t = (np.arange(nmax)[None, :] + u) * h
        ok = t < LL[:, None]
        pts = pp[:, None, :] + t[..., None] * dd[:, None, :]
        idx = np.floor((pts - lo) / vox).astype(np.int64)
        idx = np.clip(idx, 0, dims - 1)
        val = mu[idx[..., 2], idx[..., 1], idx[..., 0]]
        tau[s:s + 4000] = h * np.where(ok, val, 0.0).sum(1)
    return tau


def _unscattered_escape(rec, k):
    return ((rec["n_compton"][:, k] + rec["n_rayleigh"][:, k]) == 0) & \
        (rec["status"][:, k] != oracle.ABSORBED) & (rec["status"][:, k] != oracle.STEP_LIMIT)


@pytest.mark.parametrize("material,density", [(W.MAT_WATER, 1.3), (W.MAT_BONE, 1.9)])
def test_uniform_box_survival_matches_independent_integral(material, density):
    """Point-like source at the centre of a uniform box: the
    fraction of photons leaving unscattered equals E[exp(-mu l)] over
    isotropic directions, l the exact ray-box distance; the fraction of
    true coincidences equals E[exp(-mu (l+ + l-)) 1{both hit}]."""
    mats = W.standard_materials()
    ph = W.phantom_uniform_box(dims=(32, 32, 16), voxel=(4.0, 4.0, 4.0), material=material,
                               density=density)
    sc = W.scanner_tiny()
    n = 100_000
    r = oracle.simulate(sc, mats, ph, None, 21, 0, n, threads=8, records=True, bin_mask=3)
    rec = r["rec"]
    mt = mats[material]
    mu = density * (mt.compton[511] + mt.rayleigh[511] + mt.photo[511]) / 10.0
    rng = np.random.default_rng(123)
    m = 2_000_000
    p = rng.uniform(-4.0, 4.0, size=(m, 3))
    c = rng.uniform(-1, 1, m)
    phi = rng.uniform(0, 2 * math.pi, m)
    s = np.sqrt(1 - c * c)
    d = np.stack([s * np.cos(phi), s * np.sin(phi), c], 1)
    lo, hi = np.array([-64.0, -64.0, -32.0]), np.array([64.0, 64.0, 32.0])
    lp, lm = _box_exit(p, d, lo, hi), _box_exit(p, -d, lo, hi)
    expect_single = np.exp(-mu * lp).mean()
    got_single = np.concatenate([_unscattered_escape(rec, 0), _unscattered_escape(rec, 1)]).mean()
    sd = math.sqrt(expect_single * (1 - expect_single) / (2 * n)) * 1.5
    assert abs(got_single - expect_single) < 4 * sd
    # both photons reach the detector (axial half length 32 mm, R 310 mm)
    def zhit(pt, dd):
        a = dd[:, 0] ** 2 + dd[:, 1] ** 2
        b = pt[:, 0] * dd[:, 0] + pt[:, 1] * dd[:, 1]
        cc = pt[:, 0] ** 2 + pt[:, 1] ** 2 - 310.0**2
        t = (-b + np.sqrt(b * b - a * cc)) / a
        return pt[:, 2] + t * dd[:, 2]
    ok = (np.abs(zhit(p, d)) < 32.0) & (np.abs(zhit(p, -d)) < 32.0)
    expect_true = (np.exp(-mu * (lp + lm)) * ok).mean()
    got_true = (r["cls"] == oracle.TRUE).mean()
    sd = math.sqrt(expect_true * (1 - expect_true) / n)
    assert abs(got_true - expect_true) < 4 * sd


def _slabs():
    """Water / bone / lung slabs along x with activity everywhere."""
    ph = W.phantom_uniform_box(dims=(48, 40, 24), voxel=(5.0, 5.0, 5.0), source="uniform")
    ph.material[:, :, :16] = W.MAT_WATER
    ph.density[:, :, :16] = 1.0
    ph.material[:, :, 16:32] = W.MAT_BONE
    ph.density[:, :, 16:32] = 1.9
    ph.material[:, :, 32:] = W.MAT_LUNG
    ph.density[:, :, 32:] = 0.3
    return ph


@pytest.mark.parametrize("which", ["torso", "slabs"])
def test_heterogeneous_survival_matches_exact_ray_sums(which):
    """Torso with lungs (0.3 g/cc) and bone (1.9 g/cc), and water/bone/lung
    slabs: per photon, the unscattered-escape indicator has the same mean as
    exp(-optical depth) along its initial ray (paired comparison)."""
    mats = W.standard_materials()
    if which == "torso":
        ph = W.phantom_torso(dims=(64, 64, 32), voxel=(4.68, 4.68, 5.56))
    else:
        ph = _slabs()
    sc = W.scanner_signa()
    n = 50_000
    rec = oracle.simulate(sc, mats, ph, None, 77, 0, n, threads=8, records=True)["rec"]
    mu = _mu511(mats, ph)
    p = np.concatenate([rec["emit"], rec["emit"]])
    d = np.concatenate([rec["dir"], -rec["dir"]])
    ind = np.concatenate([_unscattered_escape(rec, 0), _unscattered_escape(rec, 1)])
    tau = _optical_depth(p, d, mu, ph)
    diff = ind - np.exp(-tau)
    assert abs(diff.mean()) < 4 * diff.std() / math.sqrt(diff.size)
    assert 0.1 < ind.mean() < 0.9


def test_vacuum_photons_fly_straight_to_analytic_hits():
    """With no attenuating matter every photon flies straight: hit points,
    crystals, rings, path lengths and TOF coordinate follow analytically."""
    sc = W.scanner_tiny()
    ph = W.phantom_uniform_box(dims=(20, 20, 10), voxel=(5.0, 5.0, 5.0),
                               material=W.MAT_VACUUM, density=0.0, source="uniform")
    n = 20_000
    r = oracle.simulate(sc, W.standard_materials(), ph, None, 4, 0, n, threads=4,
                        records=True, bin_mask=2)
    rec = r["rec"]
    assert np.all(rec["n_compton"] == 0) and np.all(rec["n_rayleigh"] == 0)
    assert np.all(rec["cls"] != oracle.SCATTER)
    R, half = sc.radius, 0.5 * sc.length
    for k, sg in ((0, 1.0), (1, -1.0)):
        p, d = rec["emit"], sg * rec["dir"]
        a = d[:, 0] ** 2 + d[:, 1] ** 2
        b = 2 * (p[:, 0] * d[:, 0] + p[:, 1] * d[:, 1])
        c = p[:, 0] ** 2 + p[:, 1] ** 2 - R * R
        t = (-b + np.sqrt(b * b - 4 * a * c)) / (2 * a)
        hit = p + t[:, None] * d
        det = rec["status"][:, k] == oracle.DETECTED
        lost = rec["status"][:, k] == oracle.LOST_AXIAL
        assert np.all(det | lost)
        np.testing.assert_array_equal(lost, ~((hit[:, 2] >= -half) & (hit[:, 2] < half)))
        np.testing.assert_allclose(rec["hit"][det, k], hit[det], atol=1e-9)
        np.testing.assert_allclose(rec["path"][det, k], t[det], rtol=1e-12)
        ang = np.mod(np.arctan2(hit[:, 1], hit[:, 0]), 2 * np.pi)
        np.testing.assert_array_equal(rec["crystal"][det, k],
                                      np.floor(ang[det] / (2 * np.pi) * sc.n_crystals).astype(int))
        np.testing.assert_array_equal(rec["ring"][det, k],
                                      np.floor((hit[det, 2] + half) / sc.ring_pitch).astype(int))
        # incidence angles: the straight ray from p hits with sin(alpha) =
        # (n x d).z where n is the radial unit vector at the hit
        nrm = hit[:, :2] / R
        sin_a = nrm[:, 0] * d[:, 1] - nrm[:, 1] * d[:, 0]
        dn = (nrm * d[:, :2]).sum(1)
        np.testing.assert_allclose(np.sin(np.radians(rec["alpha"][det, k])),
                                   sin_a[det] / np.hypot(sin_a[det], dn[det]), atol=1e-12)
    both = (r["cls"] == oracle.TRUE)
    assert both.sum() > 1000
    a_is_1 = rec["crystal"][:, 0] < rec["crystal"][:, 1]
    la = np.where(a_is_1, rec["path"][:, 0], rec["path"][:, 1])
    lb = np.where(a_is_1, rec["path"][:, 1], rec["path"][:, 0])
    np.testing.assert_allclose(rec["delta"][both], 0.5 * (la - lb)[both], rtol=1e-12)
    # (l_a - l_b)/2 is the signed distance of the emission point from the
    # LOR midpoint, towards crystal b
    ha = np.where(a_is_1[:, None], rec["hit"][:, 0], rec["hit"][:, 1])
    hb = np.where(a_is_1[:, None], rec["hit"][:, 1], rec["hit"][:, 0])
    u = (hb - ha) / np.linalg.norm(hb - ha, axis=1, keepdims=True)
    s = ((rec["emit"] - 0.5 * (ha + hb)) * u).sum(1)
    np.testing.assert_allclose(rec["delta"][both], s[both], atol=1e-9)


def test_invariants_tiny_configuration():
    sc = W.scanner_tiny()
    lut = W.lut_tiny(sc)
    n = 200_000
    r = oracle.simulate(sc, W.standard_materials(), W.phantom_water_cylinder(), lut, 12345, 0, n,
                        threads=8, records=True, acc=True)
    rec, cls = r["rec"], r["cls"]
    assert r["counts"].sum() == n                           # every history classified once
    np.testing.assert_array_equal(np.bincount(cls, minlength=8), r["counts"])
    det = (cls == oracle.TRUE) | (cls == oracle.SCATTER)
    assert det.sum() <= n                                   # never more events than histories
    assert np.all(rec["key"][~det] == -1) and np.all(rec["key"][det] >= 0)
    w = r["w"][det]
    assert np.all((w >= 0.2 * 0.2 - 1e-12) & (w <= 1.0))
    np.testing.assert_array_equal(r["q"][det], np.rint(w * 2.0**32).astype(np.int64))
    for k in range(2):
        dk = rec["status"][:, k] == oracle.DETECTED
        assert np.all(np.abs(rec["alpha"][dk, k]) < 90) and np.all(np.abs(rec["beta"][dk, k]) < 90)
        assert np.all(rec["energy"][dk, k] >= sc.e_lo)
    sc_mask = cls == oracle.SCATTER
    assert np.all((rec["n_compton"] + rec["n_rayleigh"]).sum(1)[sc_mask] > 0)
    assert np.all((rec["n_compton"] + rec["n_rayleigh"]).sum(1)[cls == oracle.TRUE] == 0)
    # the accumulator holds exactly the scatter events' weights
    expect = np.zeros(sc.n_bins, np.int64)
    np.add.at(expect, r["key"][sc_mask], r["q"][sc_mask])
    np.testing.assert_array_equal(r["acc"].ravel(), expect)


def test_same_crystal_and_out_of_range_classes():
    """Both photons detected: same transaxial crystal -> SAME_CRYSTAL, else a
    bin or OUT_OF_RANGE (coarse 16-crystal ring, 3 TOF bins, dense water)."""
    sc = W.scanner_small(n_crystals=16, n_rings=4, n_tof=3, tof_bin_mm=20.0, radius=120.0,
                         e_lo=150.0)
    ph = W.phantom_uniform_box(dims=(20, 20, 8), voxel=(4.0, 4.0, 4.0), density=2.0,
                               source="uniform")
    r = oracle.simulate(sc, W.standard_materials(), ph, None, 3, 0, 100_000, threads=8,
                        records=True)
    rec, cls = r["rec"], r["cls"]
    both = (rec["status"] == oracle.DETECTED).all(1)
    same = both & (rec["crystal"][:, 0] == rec["crystal"][:, 1])
    det = (cls == oracle.TRUE) | (cls == oracle.SCATTER)
    assert same.sum() > 10 and (cls == oracle.OUT_OF_RANGE).sum() > 50
    np.testing.assert_array_equal(cls == oracle.SAME_CRYSTAL, same)
    np.testing.assert_array_equal(both & ~same, det | (cls == oracle.OUT_OF_RANGE))
    assert np.all(np.abs(rec["delta"][cls == oracle.OUT_OF_RANGE]) >= 30.0)


def test_unit_lut_reduces_to_counts():
    """Without a LUT every coincidence adds one count (Sec. 2.2.1): a LUT of
    ones gives the same sinogram, equal to the count sinogram times 2^32."""
    sc = W.scanner_tiny()
    ph = W.phantom_water_cylinder()
    mats = W.standard_materials()
    ones = W.lut_tiny(sc)
    ones.data[:] = 1.0
    a = oracle.simulate(sc, mats, ph, None, 9, 0, 100_000, threads=8, acc=True)
    b = oracle.simulate(sc, mats, ph, ones, 9, 0, 100_000, threads=8, acc=True)
    np.testing.assert_array_equal(a["acc"], b["acc"])
    m = a["cls"] == oracle.SCATTER
    counts = np.bincount(a["key"][m], minlength=sc.n_bins)
    np.testing.assert_array_equal(a["acc"].ravel(), counts.astype(np.int64) << 32)


def test_centred_cylinder_is_symmetric():
    """A centred water cylinder on a centred grid is invariant under a 90
    degree rotation (crystal c -> c + N/4) and the z mirror (ring r ->
    n_rings - 1 - r): detected-scatter singles per crystal / ring agree."""
    sc = W.scanner_tiny()
    r = oracle.simulate(sc, W.standard_materials(), W.phantom_water_cylinder(), None, 31, 0,
                        1_000_000, threads=8, records=True)["rec"]
    sel = r["cls"] == oracle.SCATTER
    cr = np.concatenate([r["crystal"][sel, 0], r["crystal"][sel, 1]])
    rg = np.concatenate([r["ring"][sel, 0], r["ring"][sel, 1]])
    hc = np.bincount(cr, minlength=288).reshape(4, 72)
    hr = np.bincount(rg, minlength=16)
    res = stats.chi2_contingency(hc)
    assert res.pvalue > 0.01
    A, B = hr[:8], hr[::-1][:8]
    chi2 = ((A - B) ** 2 / (A + B)).sum()
    assert stats.chi2.sf(chi2, 8) > 0.01


def _small_long_scanner():
    """16 crystals x 4 rings of 40 mm, 5 TOF bins: few bins (9600), so a
    few million histories give tens of counts per bin."""
    return (W.scanner_small(n_crystals=16, n_rings=4, n_tof=5, ring_pitch=40.0, e_lo=350.0),
            W.phantom_water_cylinder(dims=(32, 32, 16), voxel=(4.0, 4.0, 4.0), radius=60.0))


def test_independent_seeds_pass_per_bin_poisson_chi_square():
    """Independent seeds give scatter count sinograms whose every bin is a
    Poisson count of the same mean: the per-bin two-sample chi-square over
    the bins with counts (tests/poisson.py) passes at p > 0.01 on a small
    scanner with tens of counts per bin and on the tiny configuration, where
    most bins hold 0 or 1 counts and the exact-moment form decides."""
    from poisson import assert_same_poisson_means, per_bin_poisson
    mats = W.standard_materials()
    for (sc, ph), n in ((_small_long_scanner(), 4_000_000),
                        ((W.scanner_tiny(), W.phantom_water_cylinder()), 1_000_000)):
        out = []
        for seed in (1001, 2002):
            r = oracle.simulate(sc, mats, ph, None, seed, 0, n, threads=8)
            m = r["cls"] == oracle.SCATTER
            out.append(np.bincount(r["key"][m], minlength=sc.n_bins))
        res = assert_same_poisson_means(*out)
        assert res["bins"] > 3000
    assert res["mean_count"] < 2.0                   # the tiny configuration: low counts
    # the same stream twice agrees too well and fails the two-sided form
    assert per_bin_poisson(out[0], out[0])["p_z"] < 1e-6
