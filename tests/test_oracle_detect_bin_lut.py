"""Oracle pins: detection of hand-built rays, LOR/TOF binning by brute force
against the continuous geometry, the multilinear 5D LUT, and the paper's
printed scanner parameters."""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_signa_configuration_matches_paper_parameters():
    g = {}
    with open(os.path.join(GOLDEN, "signa_geometry.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                g[k] = float(v)
    sc = W.scanner_signa()
    assert g["modules_per_ring"] * g["crystals_per_module_transaxial"] == sc.n_crystals
    assert g["blocks_axial"] * g["crystals_per_block_axial"] == sc.n_rings
    assert sc.module_t == g["crystals_per_module_transaxial"]
    assert sc.module_a == g["crystals_per_block_axial"]
    assert abs(sc.length - g["axial_length_mm"]) < 1e-9
    assert sc.radius == g["radius_mm"]
    assert sc.e_lo == g["lut_energy_window_lo_kev"] and sc.e_hi == g["energy_window_hi_kev"]
    t = W.scanner_tiny()
    assert t.e_lo == g["energy_window_lo_kev"] and t.e_hi == g["energy_window_hi_kev"]


# --------------------------------------------------------------------------
# detection
# --------------------------------------------------------------------------
@pytest.mark.parametrize("phi_deg", [0.3, 44.9, 90.1, 179.0, 181.0, 269.9, 359.9])
def test_radial_ray_from_centre(phi_deg):
    sc = W.scanner_tiny()
    ph = math.radians(phi_deg)
    st, cr, rg, hit, al, be, dist = oracle.detect(sc, [0, 0, 1.0], [math.cos(ph), math.sin(ph), 0])
    assert st == oracle.DETECTED
    assert cr == int(phi_deg / 360.0 * 288)
    assert rg == 8                                 # z = 1 mm -> ring 8 of 16 (4 mm pitch)
    np.testing.assert_allclose(hit[:2], [310 * math.cos(ph), 310 * math.sin(ph)], atol=1e-9)
    assert abs(al) < 1e-9 and abs(be) < 1e-9 and abs(dist - 310.0) < 1e-9


@pytest.mark.parametrize("x0", [-200.0, -50.0, 0.0, 120.0, 250.0])
def test_transaxial_incidence_angle(x0):
    """Ray along +y from (x0, 0): hits at (x0, sqrt(R^2 - x0^2)), incidence
    angle asin(x0 / R) (sign: positive towards +t = z x n)."""
    sc = W.scanner_tiny()
    st, cr, rg, hit, al, be, dist = oracle.detect(sc, [x0, 0, 0], [0, 1, 0])
    assert st == oracle.DETECTED
    np.testing.assert_allclose(hit, [x0, math.sqrt(310**2 - x0**2), 0.0], atol=1e-9)
    assert abs(al - math.degrees(math.asin(x0 / 310.0))) < 1e-9
    assert abs(be) < 1e-12


@pytest.mark.parametrize("b_deg", [-5.0, -1.0, 2.5, 5.5])
def test_axial_incidence_angle_and_axial_loss(b_deg):
    sc = W.scanner_tiny()                          # axial half length 32 mm
    b = math.radians(b_deg)
    st, cr, rg, hit, al, be, dist = oracle.detect(sc, [0, 0, 0], [0, math.cos(b), math.sin(b)])
    z = 310.0 * math.tan(b)
    if abs(z) < 32.0:
        assert st == oracle.DETECTED and abs(be - b_deg) < 1e-9
        assert rg == int(math.floor((z + 32.0) / 4.0))
    else:
        assert st == oracle.LOST_AXIAL


def test_energy_window_and_axis_parallel_ray():
    sc = W.scanner_tiny()
    assert oracle.detect(sc, [0, 0, 0], [1, 0, 0], e=424.9)[0] == oracle.ENERGY_WINDOW
    assert oracle.detect(sc, [0, 0, 0], [1, 0, 0], e=425.0)[0] == oracle.DETECTED
    assert oracle.detect(sc, [0, 0, 0], [0, 0, 1])[0] == oracle.LOST_AXIAL


# --------------------------------------------------------------------------
# binning: brute force over all crystal pairs against continuous geometry
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [16, 18, 288])
def test_lor_bins_against_continuous_geometry(N):
    sc = W.scanner_small(n_crystals=N, n_rings=3, n_tof=5)
    R = sc.radius
    seen = {}
    geo = {}
    for a in range(N):
        for b in range(a + 1, N):
            st, plane, view, rad, tof, key = oracle.bin_lor(sc, a, b, 0, 0, 0.0)
            assert st == oracle.SCATTER
            assert 0 <= view < N // 2 and 0 <= rad < N - 1
            assert (view, rad) not in seen, "two LORs share one bin"
            seen[(view, rad)] = (a, b)
            pa = R * np.array([math.cos(2 * math.pi * (a + 0.5) / N), math.sin(2 * math.pi * (a + 0.5) / N)])
            pb = R * np.array([math.cos(2 * math.pi * (b + 0.5) / N), math.sin(2 * math.pi * (b + 0.5) / N)])
            u = (pb - pa) / np.linalg.norm(pb - pa)
            nrm = np.array([-u[1], u[0]])
            # view v holds the normal angles pi(2v+1)/N and pi(2v+2)/N; orient
            # the normal towards the view's nominal direction
            ref = math.pi * (2 * view + 1.5) / N
            if nrm @ np.array([math.cos(ref), math.sin(ref)]) < 0:
                nrm = -nrm
            psi = math.atan2(nrm[1], nrm[0])
            psi = ref + math.remainder(psi - ref, 2 * math.pi)
            geo[(view, rad)] = (psi, float(nrm @ pa), ref)
    assert len(seen) == N * (N - 1) // 2               # bijection onto views x radial bins
    for v in range(N // 2):
        for r in range(N - 1):
            psi, rho, ref = geo[(v, r)]
            # each LOR's normal is one of the view's two interleaved angles
            assert abs(psi - ref) < 0.5 * math.pi / N + 1e-9
        rhos = [geo[(v, r)][1] for r in range(N - 1)]
        # radial index is monotone in the signed distance from the centre
        dr = np.diff(rhos)
        assert np.all(dr > 0) or np.all(dr < 0)
        # the centre LOR (a diameter) sits at radial index N/2 - 1
        assert abs(rhos[N // 2 - 1]) < 1e-9


def test_tof_and_plane_indexing():
    sc = W.scanner_small(n_crystals=16, n_rings=4, n_tof=5, tof_bin_mm=40.0)
    # bin t covers delta in [(t - 2.5) * 40, (t - 1.5) * 40)
    for delta, t in [(-100.0, 0), (-60.0, 1), (-20.0, 2), (19.9, 2), (20.0, 3), (99.9, 4)]:
        st, plane, view, rad, tof, key = oracle.bin_lor(sc, 1, 9, 2, 3, delta)
        assert st == oracle.SCATTER and tof == t and plane == 2 * 4 + 3
        assert key == ((plane * 8 + view) * 15 + rad) * 5 + tof
    for delta in (-100.1, 100.0):
        assert oracle.bin_lor(sc, 1, 9, 0, 0, delta)[0] == oracle.OUT_OF_RANGE


def test_radial_clip_is_centred():
    full = W.scanner_small(n_crystals=16)
    clip = W.scanner_small(n_crystals=16, n_rad=9)
    for a in range(16):
        for b in range(a + 1, 16):
            r_full = oracle.bin_lor(full, a, b, 0, 0, 0.0)[3]
            st, _, _, r, _, _ = oracle.bin_lor(clip, a, b, 0, 0, 0.0)
            if 3 <= r_full < 12:
                assert st == oracle.SCATTER and r == r_full - 3
            else:
                assert st == oracle.OUT_OF_RANGE


# --------------------------------------------------------------------------
# 5D LUT
# --------------------------------------------------------------------------
def _lut(n_e=5, n_a=4, n_b=3, n_t=2, n_z=3, f=None):
    e_min, e_max = 425.0, 511.0
    ec = e_min + (np.arange(n_e) + 0.5) * (e_max - e_min) / n_e
    ac = -90 + (np.arange(n_a) + 0.5) * 180.0 / n_a
    bc = -90 + (np.arange(n_b) + 0.5) * 180.0 / n_b
    Z, T, E, A, B = np.meshgrid(np.arange(n_z), np.arange(n_t), ec, ac, bc, indexing="ij")
    data = f(E, A, B, T, Z).astype(np.float32)
    return W.Lut(n_e, e_min, e_max, n_a, n_b, n_t, n_z, data), ec, ac, bc


def _multilinear(E, A, B, T, Z):
    # multilinear in (E, A, B) with coefficients depending on (T, Z);
    # small integers keep every value exact in float32
    return (3 + T + 2 * Z + 0.25 * (E - 425) - 0.5 * A + 0.75 * B
            + 0.01 * (E - 425) * A - 0.02 * A * B + 0.003 * (E - 425) * B
            + 0.0001 * (E - 425) * A * B * (1 + T))


def test_lut_node_values():
    lut, ec, ac, bc = _lut(f=lambda E, A, B, T, Z: 1 + E * 0 + 7 * A + B + 100 * T + 1000 * Z)
    for z in range(3):
        for t in range(2):
            for i, e in enumerate(ec):
                for j, a in enumerate(ac):
                    for k, b in enumerate(bc):
                        assert oracle.lut_prob(lut, e, a, b, t, z) == pytest.approx(
                            float(lut.data[z, t, i, j, k]), rel=1e-12)


def test_lut_reproduces_multilinear_functions_and_clamps():
    lut, ec, ac, bc = _lut(f=_multilinear)
    rng = np.random.default_rng(0)
    for _ in range(500):
        e = rng.uniform(ec[0], ec[-1])
        a = rng.uniform(ac[0], ac[-1])
        b = rng.uniform(bc[0], bc[-1])
        t, z = int(rng.integers(2)), int(rng.integers(3))
        assert oracle.lut_prob(lut, e, a, b, t, z) == pytest.approx(_multilinear(e, a, b, t, z),
                                                                    rel=1e-6, abs=1e-6)
    # outside the outer nodes the value is held (clamped coordinates)
    for e, a, b in [(300.0, -89.0, 80.0), (600.0, 89.9, -89.9), (430.0, 0.0, 89.0)]:
        ee, aa, bb = np.clip(e, ec[0], ec[-1]), np.clip(a, ac[0], ac[-1]), np.clip(b, bc[0], bc[-1])
        assert oracle.lut_prob(lut, e, a, b, 1, 2) == pytest.approx(_multilinear(ee, aa, bb, 1, 2),
                                                                    rel=1e-6, abs=1e-6)


def test_lut_degenerate_axes_and_no_lut():
    # one bin on an axis = constant along it (lower-dimensional LUTs)
    lut, ec, ac, bc = _lut(n_a=1, n_b=1, f=lambda E, A, B, T, Z: 0.5 + 0.001 * (E - 425) + 0 * A)
    for a, b in [(-80.0, 10.0), (0.0, 0.0), (85.0, -60.0)]:
        assert oracle.lut_prob(lut, 470.0, a, b, 0, 0) == pytest.approx(0.5 + 0.001 * 45, rel=1e-6)
    assert oracle.lut_prob(None, 470.0, 10.0, 10.0, 0, 0) == 1.0


def _lut_copy(lut, data):
    return W.Lut(lut.n_e, lut.e_min, lut.e_max, data.shape[3], data.shape[4], data.shape[1], data.shape[0],
                 np.ascontiguousarray(data, dtype=np.float32), lut.a_min, lut.a_max, lut.b_min, lut.b_max)


def test_lower_dimensional_lut_equals_full_lut_constant_on_dropped_axes():
    """Sec. 2.2.2's lower-dimensional LUTs: a LUT with one bin on the
    position axes gives every history the weight of the full-size LUT whose
    values repeat that bin at every position (bit for bit: the same entries
    are read), and one bin on the angle axes that of a full LUT constant in
    angle (up to the rounding of the multilinear weights)."""
    sc = W.scanner_tiny()
    mats, ph = W.standard_materials(), W.phantom_water_cylinder()
    lut = W.lut_tiny(sc)
    n = 50_000
    red_pos = _lut_copy(lut, lut.data[:1, :1])
    full_pos = _lut_copy(lut, np.broadcast_to(lut.data[:1, :1], lut.data.shape))
    a = oracle.simulate(sc, mats, ph, red_pos, 9, 0, n, threads=8)
    b = oracle.simulate(sc, mats, ph, full_pos, 9, 0, n, threads=8)
    assert (a["key"] >= 0).sum() > 200
    np.testing.assert_array_equal(a["q"], b["q"])
    np.testing.assert_array_equal(a["key"], b["key"])
    red_ang = _lut_copy(lut, lut.data[:, :, :, 3:4, 5:6])
    full_ang = _lut_copy(lut, np.broadcast_to(lut.data[:, :, :, 3:4, 5:6], lut.data.shape))
    a = oracle.simulate(sc, mats, ph, red_ang, 9, 0, n, threads=8)
    b = oracle.simulate(sc, mats, ph, full_ang, 9, 0, n, threads=8)
    m = a["key"] >= 0
    np.testing.assert_allclose(a["w"][m], b["w"][m], rtol=1e-12)
    # and the reduced LUT differs from the full one where the full one varies
    c = oracle.simulate(sc, mats, ph, lut, 9, 0, n, threads=8)
    assert not np.allclose(a["w"][m], c["w"][m])


def test_reduced_lut_is_the_ratio_of_summed_histograms():
    """The energy-only and energy+crystal LUTs made from the two histograms
    equal the ratio of explicit sums over the dropped axes, and the reduced
    LUT is a detection probability where photons arrived."""
    sc = W.scanner_tiny()
    lut = W.lut_tiny(sc)
    inc, det = W.lut_histograms(lut, counts=5.0)
    e_only = W.lut_reduced(lut, inc, det, keep=("e",))
    assert e_only.data.shape == (1, 1, lut.n_e, 1, 1)
    for ie in (0, 7, lut.n_e - 1):
        num = sum(int(det[z, t, ie, i, j]) for z in range(lut.n_apos) for t in range(lut.n_tpos)
                  for i in range(lut.n_a) for j in range(lut.n_b))
        den = sum(int(inc[z, t, ie, i, j]) for z in range(lut.n_apos) for t in range(lut.n_tpos)
                  for i in range(lut.n_a) for j in range(lut.n_b))
        assert e_only.data[0, 0, ie, 0, 0] == np.float32(num / den)
    e_pos = W.lut_reduced(lut, inc, det, keep=("e", "t", "z"))
    assert e_pos.data.shape == (lut.n_apos, lut.n_tpos, lut.n_e, 1, 1)
    z, t, ie = 1, 2, 3
    num = int(det[z, t, ie].sum())
    den = int(inc[z, t, ie].sum())
    assert e_pos.data[z, t, ie, 0, 0] == np.float32(num / den)
    assert e_pos.data.min() >= 0.0 and e_pos.data.max() <= 1.0
