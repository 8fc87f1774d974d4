"""Oracle pins for the energy-resolution variant (the no-LUT mode of Sec.
2.2.1: 11.2 % resolution, 425-650 keV window).  The detected energy is the
photon energy plus sigma(E) g with sigma(E) = r sqrt(511 E) / 2.3548 (FWHM
r * 511 keV at 511 keV, scaling as sqrt(E)); the window tests it."""
import math

import numpy as np
from scipy import stats

import oracle
import workloads as W

R = 0.112
FWHM_TO_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))


def sigma(e):
    return R * np.sqrt(511.0 * e) / FWHM_TO_SIGMA


def scanner(lo=425.0, hi=650.0):
    sc = W.scanner_tiny()
    sc.e_lo, sc.e_hi, sc.e_res = lo, hi, R
    return sc


def test_unscattered_photons_are_blurred_by_the_511_kev_resolution():
    """Vacuum: every photon arrives with 511 keV; (E_det - 511) / sigma(511)
    is standard normal, and a narrow window keeps the normal fraction."""
    ph = W.phantom_uniform_box(dims=(16, 16, 8), material=W.MAT_VACUUM, density=0.0)
    sc = scanner(490.0, 530.0)
    r = oracle.simulate(sc, W.standard_materials(), ph, None, 31, 0, 60_000, threads=8, records=True)
    rec = r["rec"]
    hit = rec["status"][:, 0] != oracle.LOST_AXIAL
    assert np.all(rec["energy"][hit, 0] == 511.0)
    z = (rec["e_det"][hit, 0] - 511.0) / sigma(511.0)
    assert stats.kstest(z, "norm").pvalue > 0.01
    p = stats.norm.cdf(19.0 / sigma(511.0)) - stats.norm.cdf(-21.0 / sigma(511.0))
    kept = (rec["status"][hit, 0] == oracle.DETECTED).mean()
    n = hit.sum()
    assert abs(kept - p) < 4.0 * math.sqrt(p * (1 - p) / n)


def test_blur_scales_with_sqrt_energy_and_window_uses_blurred_energy():
    """Water: scattered photons of every energy have standard-normal
    residuals (E_det - E) / sigma(E); the window decision follows E_det, so
    photons below 425 keV are detected and photons inside can be rejected."""
    sc = scanner()
    r = oracle.simulate(sc, W.standard_materials(), W.phantom_water_cylinder(), None, 32, 0, 120_000,
                        threads=8, records=True)
    rec = r["rec"]
    st, e, ed = rec["status"].ravel(), rec["energy"].ravel(), rec["e_det"].ravel()
    # photons that reached the detector (one dropped in transport has no detected energy)
    tested = ((st == oracle.DETECTED) | (st == oracle.ENERGY_WINDOW)) & (ed != 0.0)
    scat = tested & (e < 505.0)
    assert scat.sum() > 2000
    z = (ed[scat] - e[scat]) / sigma(e[scat])
    assert stats.kstest(z, "norm").pvalue > 0.01
    det = st == oracle.DETECTED
    assert np.all((ed[det] >= 425.0) & (ed[det] <= 650.0))
    assert np.any(det & (e < 425.0))
    assert np.any((st == oracle.ENERGY_WINDOW) & (e >= 425.0) & (ed < 425.0))


def test_compton_photons_are_dropped_only_five_sigma_below_the_window():
    """A photon scattering below e_lo - 5 sigma(e_lo) ends there (it could
    be blurred into the window with probability < 3e-7); none detected is
    that low, and some photons between that cut and e_lo are still tracked."""
    sc = scanner()
    cut = 425.0 - 5.0 * sigma(425.0)
    r = oracle.simulate(sc, W.standard_materials(), W.phantom_water_cylinder(), None, 33, 0, 60_000,
                        threads=8, records=True)
    rec = r["rec"]
    st, e = rec["status"].ravel(), rec["energy"].ravel()
    assert np.all(e[st == oracle.DETECTED] >= cut)
    dropped = (st == oracle.ENERGY_WINDOW) & (e < cut)
    assert dropped.sum() > 100
    # photons ended in transport (no hit on the cylinder) are all below the cut
    in_transport = (st == oracle.ENERGY_WINDOW) & np.all(rec["hit"].reshape(-1, 3) == 0.0, axis=1)
    assert in_transport.sum() > 100 and np.all(e[in_transport] < cut)
    assert np.any((st != oracle.ENERGY_WINDOW) & (e >= cut) & (e < 425.0))
