"""Oracle pins for gaps between detector modules and blocks (Sec. 2.2.1-2.2.2):
module/block placement of hits with virtual crystals in the half gaps, the
edge-crystal assignment probability, and its use in the simulation."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def gapped(mode=2):
    return W.scanner_signa_gaps(gap_mode=mode)


def _hit(sc, phi, z):
    return np.array([sc.radius * math.cos(phi), sc.radius * math.sin(phi), z])


def test_transaxial_placement_of_crystals_and_half_gaps():
    sc = gapped()
    n_mod = sc.n_crystals // sc.module_t
    Phi = 2 * math.pi / n_mod
    gamma = sc.gap_t / sc.radius
    cw = (Phi - gamma) / sc.module_t
    for m in (0, 5, n_mod - 1):
        for j in (0, 7, sc.module_t - 1):
            fl, tp, _, cr, _, _, _, _, _ = oracle.place(sc, _hit(sc, m * Phi + gamma / 2 + (j + 0.5) * cw, 1.0))
            assert (fl & 1) == 0 and tp == j + 1 and cr == m * sc.module_t + j
        fl, tp, _, cr, _, xt, _, bt, _ = oracle.place(sc, _hit(sc, m * Phi + 0.3 * gamma / 2, 1.0))
        assert fl & 1 and tp == 0 and bt == m and cr == -1
        assert abs(xt - 0.3 * sc.gap_t / 2) < 1e-9
        fl, tp, _, _, _, xt, _, bt, _ = oracle.place(sc, _hit(sc, (m + 1) * Phi - 0.6 * gamma / 2, 1.0))
        assert fl & 1 and tp == sc.module_t + 1 and bt == m + 1
        assert abs(xt + 0.6 * sc.gap_t / 2) < 1e-9


def test_axial_placement_of_rings_and_half_gaps():
    sc = gapped()
    L = sc.n_rings * sc.ring_pitch
    n_blk = sc.n_rings // sc.module_a
    P = L / n_blk
    rw = (P - sc.gap_a) / sc.module_a
    for b in range(n_blk):
        for j in (0, sc.module_a - 1):
            z = -L / 2 + b * P + sc.gap_a / 2 + (j + 0.5) * rw
            fl, tp, ap, _, rg, _, _, _, _ = oracle.place(sc, _hit(sc, 0.1, z))
            assert (fl & 2) == 0 and rg == b * sc.module_a + j and ap == b * (sc.module_a + 2) + j + 1
        fl, _, ap, _, rg, _, xa, _, ba = oracle.place(sc, _hit(sc, 0.1, -L / 2 + b * P + 0.2))
        assert fl & 2 and ap == b * (sc.module_a + 2) and ba == b and rg == -1 and abs(xa - 0.2) < 1e-9


def test_uniform_hits_fall_in_gaps_at_their_area_fraction():
    sc = gapped()
    rng = np.random.default_rng(0)
    n = 20000
    phi = rng.uniform(0, 2 * math.pi, n)
    z = rng.uniform(-0.5, 0.5, n) * sc.n_rings * sc.ring_pitch
    fl = np.array([oracle.place(sc, _hit(sc, p, zz))[0] for p, zz in zip(phi, z)])
    ft = sc.gap_t * (sc.n_crystals // sc.module_t) / (2 * math.pi * sc.radius)
    fa = sc.gap_a * (sc.n_rings // sc.module_a) / (sc.n_rings * sc.ring_pitch)
    for frac, bit in ((ft, 1), (fa, 2)):
        got = ((fl & bit) != 0).mean()
        assert abs(got - frac) < 4 * math.sqrt(frac * (1 - frac) / n)


def _edge_prob_by_sampling(sc, x0, theta_deg, gap, n=200_000):
    """Independent evaluation: path lengths through the two blocks by
    midpoint sampling of the line over the crystal depth."""
    th = math.radians(theta_deg)
    y = (np.arange(n) + 0.5) * sc.crystal_depth / n
    x = x0 + (y - sc.doi) * math.tan(th)
    dl = sc.crystal_depth / n / math.cos(th)
    l1, l2 = (x < -gap / 2).sum() * dl, (x > gap / 2).sum() * dl
    mu = sc.mu_block
    if theta_deg > 0:
        p1 = 1 - math.exp(-mu * l1)
        p2 = math.exp(-mu * l1) * (1 - math.exp(-mu * l2))
    else:
        p2 = 1 - math.exp(-mu * l2)
        p1 = math.exp(-mu * l2) * (1 - math.exp(-mu * l1))
    return p1 / (p1 + p2) if p1 + p2 > 0 else (1.0 if x0 < 0 else 0.0)


@pytest.mark.parametrize("x0,theta", [(0.0, 30.0), (-0.7, 10.0), (0.4, -45.0), (0.9, 60.0), (-0.2, -5.0)])
def test_edge_probability_matches_path_length_model(x0, theta):
    sc = gapped()
    got = oracle.edge_prob(sc, x0, theta, 2.0)
    assert abs(got - _edge_prob_by_sampling(sc, x0, theta, 2.0)) < 2e-4


def test_edge_probability_symmetry_and_normal_incidence():
    sc = gapped()
    for x0, th in ((0.3, 20.0), (-0.8, 50.0), (0.0, 5.0)):
        assert abs(oracle.edge_prob(sc, x0, th, 2.0) + oracle.edge_prob(sc, -x0, -th, 2.0) - 1.0) < 1e-12
    assert oracle.edge_prob(sc, -0.5, 0.0, 2.0) == 1.0 and oracle.edge_prob(sc, 0.5, 0.0, 2.0) == 0.0
    # a photon meeting block 1 first at steep incidence is mostly detected there
    assert oracle.edge_prob(sc, 0.0, 60.0, 2.0) > 0.5


def _vacuum():
    return W.phantom_uniform_box(dims=(32, 32, 24), voxel=(4.0, 4.0, 4.0), material=W.MAT_VACUUM, density=0.0)


def test_gap_photons_are_lost_or_assigned_to_edge_crystals():
    """Mode 1: no detected photon lies in a gap.  Mode 2: photons in a
    transaxial gap end on one of its two edge crystals, on the negative side
    with the mean of their edge probabilities; the LUT saw the virtual
    position (a LUT that is constant per transaxial position tells)."""
    ph = _vacuum()
    n = 40_000
    r1 = oracle.simulate(gapped(1), W.standard_materials(), ph, None, 5, 0, n, threads=8, records=True)["rec"]
    sc = gapped(2)
    tpos_val = np.linspace(0.3, 1.0, sc.n_tpos).astype(np.float32)
    lut = W.lut_signa(sc)
    lut.data[:] = tpos_val[None, :, None, None, None]
    r2 = oracle.simulate(sc, W.standard_materials(), ph, lut, 5, 0, n, threads=8, records=True)["rec"]
    det1 = r1["status"] == oracle.DETECTED
    det2 = r2["status"] == oracle.DETECTED
    for k in range(2):
        for i in np.flatnonzero(det1[:, k])[:3000]:
            assert oracle.place(sc, r1["hit"][i, k])[0] == 0
    p_neg, neg, pa_low, low = [], [], [], []
    n_blk = sc.n_rings // sc.module_a
    for i in np.flatnonzero(det2[:, 0])[:20000]:
        fl, tp, ap, cr, rg, xt, xa, bt, ba = oracle.place(sc, r2["hit"][i, 0])
        assert abs(r2["prob"][i, 0] - tpos_val[tp]) < 1e-6
        if fl & 1:
            left, right = (bt * sc.module_t - 1) % sc.n_crystals, (bt * sc.module_t) % sc.n_crystals
            assert r2["crystal"][i, 0] in (left, right)
            p_neg.append(oracle.edge_prob(sc, xt, r2["alpha"][i, 0], sc.gap_t))
            neg.append(r2["crystal"][i, 0] == left)
        if fl & 2:
            ring = r2["ring"][i, 0]
            if ba == 0:
                assert ring == 0
            elif ba == n_blk:
                assert ring == sc.n_rings - 1
            else:  # an inner block gap: one of its two edge rings, the lower with p1
                assert ring in (ba * sc.module_a - 1, ba * sc.module_a)
                pa_low.append(oracle.edge_prob(sc, xa, r2["beta"][i, 0], sc.gap_a))
                low.append(ring == ba * sc.module_a - 1)
    for p, hit in ((p_neg, neg), (pa_low, low)):
        p, hit = np.array(p), np.array(hit, dtype=np.float64)
        assert p.size > 200
        var = (p * (1 - p)).sum()
        assert abs(hit.sum() - p.sum()) < 4 * math.sqrt(var) + 1
        # each photon follows its own probability: the residuals do not correlate with
        # 2p - 1 (swapping the two edges would give a sum of -(2p - 1)^2)
        c = 2 * p - 1
        z = ((hit - p) * c).sum()
        assert abs(z) < 4 * math.sqrt((p * (1 - p) * c * c).sum()) + 1
        assert (c * c).sum() > 8 * math.sqrt((p * (1 - p) * c * c).sum()) + 8
