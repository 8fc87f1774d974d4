"""Oracle pins: Compton (Klein-Nishina), Rayleigh, cross-section tables,
Compton kinematics inside the transport."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
import workloads as W


def kn_dsigma_dmu(mu, e):
    """Klein-Nishina differential cross section per unit cos(theta) (up to a
    constant): (P^2/2)(P + 1/P - sin^2), P = E'/E (textbook closed form)."""
    a = e / 511.0
    P = 1.0 / (1.0 + a * (1.0 - mu))
    return P * P * (P + 1.0 / P - (1.0 - mu * mu))


def _binned_chi2(samples, pdf, bins=40, lo=-1.0, hi=1.0):
    edges = np.linspace(lo, hi, bins + 1)
    counts = np.histogram(samples, bins=edges)[0]
    mass = np.array([integrate.quad(pdf, edges[i], edges[i + 1])[0] for i in range(bins)])
    expect = mass / mass.sum() * samples.size
    chi2 = ((counts - expect) ** 2 / expect).sum()
    return stats.chi2.sf(chi2, bins - 1)


@pytest.mark.parametrize("e", [511.0, 340.0, 200.0])
def test_compton_angles_follow_klein_nishina(e):
    c, eo = oracle.sample_compton(e, seed=17, n=200_000)
    assert np.all((c >= -1.0) & (c <= 1.0))
    assert _binned_chi2(c, lambda m: kn_dsigma_dmu(m, e)) > 0.01
    # Compton relation E' = E / (1 + (E/511)(1 - cos theta))
    np.testing.assert_allclose(eo, e / (1.0 + (e / 511.0) * (1.0 - c)), rtol=1e-12)


def test_compton_mean_energy_loss_closed_form():
    # <E'/E> under Klein-Nishina at 511 keV by quadrature vs the sample mean
    e = 511.0
    c, eo = oracle.sample_compton(e, seed=3, n=400_000)
    num = integrate.quad(lambda m: kn_dsigma_dmu(m, e) / (1 + (e / 511) * (1 - m)), -1, 1)[0]
    den = integrate.quad(lambda m: kn_dsigma_dmu(m, e), -1, 1)[0]
    mean = (eo / e).mean()
    sd = (eo / e).std() / math.sqrt(eo.size)
    assert abs(mean - num / den) < 4 * sd


def test_rayleigh_without_form_factor_is_thomson():
    c = oracle.sample_rayleigh(511.0, 0.0, seed=5, n=200_000)
    assert _binned_chi2(c, lambda m: 1.0 + m * m) > 0.01


@pytest.mark.parametrize("e,kappa", [(511.0, 500.0), (350.0, 800.0), (200.0, 30.0)])
def test_rayleigh_with_form_factor(e, kappa):
    b = kappa * (e / 511.0) ** 2
    c = oracle.sample_rayleigh(e, kappa, seed=8, n=200_000)
    pdf = lambda m: (1.0 + m * m) / (1.0 + b * (1.0 - m) / 2.0) ** 2
    # forward peaked: bins uniform in s = (1 - mu)/2 on a log-ish grid
    s_edges = np.concatenate([[0.0], np.geomspace(1e-5, 1.0, 30)])
    mu_edges = np.sort(1.0 - 2.0 * s_edges)
    counts = np.histogram(c, bins=mu_edges)[0]
    mass = np.array([integrate.quad(pdf, mu_edges[i], mu_edges[i + 1])[0]
                     for i in range(mu_edges.size - 1)])
    expect = mass / mass.sum() * c.size
    keep = expect > 5
    chi2 = ((counts[keep] - expect[keep]) ** 2 / expect[keep]).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 0.01


def test_water_attenuation_at_511():
    # Klein-Nishina total cross section: closed form vs direct quadrature of
    # the differential cross section, and mu_water(511 keV) ~ 0.096 cm^-1
    r_e = W.CLASSICAL_ELECTRON_RADIUS_CM
    a = 511.0 / W.ELECTRON_REST_KEV

    def dsig_domega(mu):
        P = 1.0 / (1.0 + a * (1.0 - mu))
        return 0.5 * r_e**2 * P * P * (P + 1.0 / P - (1.0 - mu * mu))

    quad = 2 * math.pi * integrate.quad(dsig_domega, -1, 1)[0]
    assert abs(W.klein_nishina_sigma_cm2(511.0) / quad - 1) < 1e-10
    water = W.standard_materials()[W.MAT_WATER]
    mu = water.compton[511] + water.rayleigh[511] + water.photo[511]
    assert abs(mu - 0.096) < 0.001


def test_compton_relation_inside_transport():
    """Every first Compton event in the tracked histories obeys
    E' = E/(1 + (E/511)(1 - d.d')) with d, d' the directions before/after."""
    sc = W.scanner_tiny()
    ph = W.phantom_water_cylinder()
    r = oracle.simulate(sc, W.standard_materials(), ph, None, 11, 0, 50_000, threads=8,
                        records=True)["rec"]
    m = r["c_e_before"] > 0
    assert m.sum() > 10_000
    cb = (r["c_dir_before"][m] * r["c_dir_after"][m]).sum(1)
    np.testing.assert_allclose(np.linalg.norm(r["c_dir_after"][m], axis=1), 1.0, atol=1e-12)
    eb, ea = r["c_e_before"][m], r["c_e_after"][m]
    np.testing.assert_allclose(ea, eb / (1.0 + (eb / 511.0) * (1.0 - cb)), rtol=1e-9)
    # azimuth about the incoming direction is uniform
    d0, d1 = r["c_dir_before"][m], r["c_dir_after"][m]
    ref = np.cross(d0, np.array([0.0, 0.0, 1.0]))
    ref /= np.linalg.norm(ref, axis=1, keepdims=True)
    perp = d1 - cb[:, None] * d0
    ok = np.linalg.norm(perp, axis=1) > 1e-6
    y = np.cross(d0, ref)
    phi = np.arctan2((perp * y).sum(1), (perp * ref).sum(1))[ok]
    assert stats.chisquare(np.histogram(phi, bins=24, range=(-np.pi, np.pi))[0]).pvalue > 0.01
