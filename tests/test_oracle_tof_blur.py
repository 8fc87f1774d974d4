"""Oracle pin: the Gaussian TOF blur of the paper-scale configuration.

Sec. 2.2.1 bins coincidences by the difference of the two photons' arrival
times.  A timing difference dt moves the estimated annihilation point along
the LOR by c dt / 2, so the binned coordinate is the half path difference
(l_a - l_b) / 2 (the geometric part is pinned by the vacuum-geometry test),
and a coincidence timing resolution of FWHM 400 ps (the paper-scale
configuration; Sec. 2.1 quotes 380 ps for the real scanner) blurs it by a
Gaussian of

    sigma = c * 400 ps / 2 / (2 sqrt(2 ln 2)) = 25.462 mm,  c = 0.299792458 mm/ps.

On a phantom with no attenuating matter every photon flies straight, so the
unblurred coordinate of each history follows from its recorded emission point
and direction by an independent ray-cylinder intersection.  The pins:
  * (delta - delta_geom) / sigma is standard normal (KS), with sigma the
    number above written out, not taken from the workload module;
  * the TOF-bin frequencies (and the out-of-range count) equal the normal
    integral over the bin edges, summed over the histories;
  * the blur is independent of the emission draws (no correlation with the
    emission point or direction), i.e. it reads words of its own.
A wrong FWHM-to-sigma factor, a missing 1/2 of the half path difference, a
blur on the full difference, or a blur drawn from the emission words fails
one of them.  (Box-Muller's cosine and sine branches are both standard
normal; the oracle's choice of the cosine is a convention the GPU path
follows, checked history by history in the GPU tests.)
"""
import math

import numpy as np
from scipy import stats

import oracle
import workloads as W

SIGMA_400PS_MM = 25.462027   # 0.299792458 * 400 / 2 / 2.3548200450309493


def test_configuration_sigma_is_that_of_400ps():
    assert abs(0.299792458 * 400.0 / 2.0 / (2.0 * math.sqrt(2.0 * math.log(2.0))) - SIGMA_400PS_MM) < 1e-6
    assert abs(W.scanner_signa().tof_sigma_mm - SIGMA_400PS_MM) < 1e-6


def _geometric_delta(rec, sc):
    """(l_a - l_b) / 2 of straight flights from the emission point, a the
    photon in the lower-numbered crystal (an independent intersection of each
    ray with the cylinder x^2 + y^2 = R^2)."""
    R = sc.radius
    ell = []
    for sg in (1.0, -1.0):
        p, d = rec["emit"], sg * rec["dir"]
        a = d[:, 0] ** 2 + d[:, 1] ** 2
        b = 2 * (p[:, 0] * d[:, 0] + p[:, 1] * d[:, 1])
        c = p[:, 0] ** 2 + p[:, 1] ** 2 - R * R
        ell.append((-b + np.sqrt(b * b - 4 * a * c)) / (2 * a))
    a_is_1 = rec["crystal"][:, 0] < rec["crystal"][:, 1]
    la = np.where(a_is_1, ell[0], ell[1])
    lb = np.where(a_is_1, ell[1], ell[0])
    return 0.5 * (la - lb)


def _vacuum_run(n, seed):
    sc = W.scanner_signa()
    ph = W.phantom_uniform_box(dims=(40, 40, 30), voxel=(4.0, 4.0, 4.0), material=W.MAT_VACUUM,
                               density=0.0, source="uniform")
    r = oracle.simulate(sc, W.standard_materials(), ph, None, seed, 0, n, threads=8, records=True,
                        bin_mask=2)
    rec = r["rec"]
    both = (r["cls"] == oracle.TRUE) | (r["cls"] == oracle.OUT_OF_RANGE)
    return sc, rec[both], r["cls"][both]


def test_tof_blur_is_gaussian_with_the_400ps_sigma():
    sc, rec, cls = _vacuum_run(400_000, 17)
    assert rec.size > 50_000
    assert np.all(rec["n_compton"] == 0) and np.all(rec["n_rayleigh"] == 0)
    z = (rec["delta"] - _geometric_delta(rec, sc)) / SIGMA_400PS_MM
    assert stats.kstest(z, "norm").pvalue > 0.01
    assert abs(z.mean()) < 5.0 / math.sqrt(z.size)
    assert abs(z.std() - 1.0) < 0.01
    # independent of the emission draws: no correlation with the emission
    # point or direction
    for f in (rec["emit"][:, 0], rec["emit"][:, 1], rec["emit"][:, 2], rec["dir"][:, 0], rec["dir"][:, 2]):
        assert abs(np.corrcoef(z, f)[0, 1]) < 5.0 / math.sqrt(z.size)


def test_tof_bin_frequencies_equal_the_normal_integral():
    sc, rec, cls = _vacuum_run(300_000, 23)
    g = _geometric_delta(rec, sc)
    w, nt = sc.tof_bin_mm, sc.n_tof
    edges = (np.arange(nt + 1) - 0.5 * nt) * w                      # bin t: [edges[t], edges[t+1])
    cdf = stats.norm.cdf((edges[None, :] - g[:, None]) / SIGMA_400PS_MM)
    p_bin = np.diff(cdf, axis=1)                                      # (histories, n_tof)
    expect = np.append(p_bin.sum(axis=0), (1.0 - p_bin.sum(axis=1)).sum())
    seen = np.append(np.bincount(rec["tof"][cls == oracle.TRUE], minlength=nt),
                     (cls == oracle.OUT_OF_RANGE).sum())
    assert seen.sum() == rec.size
    keep = expect > 5.0
    rest = (expect[~keep].sum(), seen[~keep].sum())
    e = np.append(expect[keep], rest[0])
    o = np.append(seen[keep], rest[1])
    chi2 = ((o - e) ** 2 / np.maximum(e, 1e-12)).sum()
    assert stats.chi2.sf(chi2, e.size - 1) > 0.01
