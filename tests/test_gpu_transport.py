"""GPU parity of the fused transport kernel against the oracle (through the
C ABI): per-history class, bin and weight on shared Philox streams, exact
int64 accumulation, launch-shape / partition / checkpoint independence,
LUT precisions, the paper-scale configuration, and edge cases."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import paper_2509_05047_gb300 as psc
import workloads as W

from gpu_helpers import Session, compare_histories, sinogram_from

pytestmark = pytest.mark.gpu

SEED = 12345


@pytest.fixture(scope="module")
def tiny():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_tiny()
    mats = W.standard_materials()
    ph = W.phantom_water_cylinder()
    lut = W.lut_tiny(sc)
    s = Session(sc, mats, ph, lut)
    s.mats, s.ph, s.lut = mats, ph, lut
    yield s
    s.close()


@pytest.mark.parametrize("first,n", [(0, 200_003), (10_000_000_000, 65_537)])
def test_tiny_histories_match_oracle(tiny, first, n):
    tiny.zero()
    g = tiny.run(SEED, first, n)
    r = oracle.simulate(tiny.sc, tiny.mats, tiny.ph, tiny.lut, SEED, first, n, threads=8)
    same = compare_histories(g, r)
    # class counters agree with the listmode
    st = g["stats"]
    np.testing.assert_array_equal([st[c] for c in psc.CLASSES], np.bincount(g["cls"], minlength=8))
    # the accumulator holds exactly the listmode's scatter weights
    acc = tiny.acc().cpu().numpy()
    np.testing.assert_array_equal(acc, sinogram_from(g["key"], g["q"], g["cls"], tiny.sc.n_bins))
    assert st["binned"] == (g["cls"] == 7).sum() and st["weight_sum"] == g["q"][g["cls"] == 7].sum()
    # class frequencies agree with the oracle's
    assert (~same).sum() <= 0.001 * n


def test_unit_lut_count_sinogram_is_bit_exact_on_matched_histories(tiny):
    """LUT = 1 (no LUT): every event adds exactly 2^32; the GPU count
    sinogram minus its mismatched histories equals the oracle's minus its
    mismatched histories, bit for bit."""
    n = 300_000
    tiny.zero()
    g = tiny.run(SEED + 1, 0, n, lut=0)
    r = oracle.simulate(tiny.sc, tiny.mats, tiny.ph, None, SEED + 1, 0, n, threads=8)
    same = compare_histories(g, r, w_rtol=0.0)
    acc = tiny.acc().cpu().numpy()
    gm = sinogram_from(g["key"][~same], g["q"][~same], g["cls"][~same], tiny.sc.n_bins)
    rm = sinogram_from(r["key"], r["q"], r["cls"], tiny.sc.n_bins) - \
        sinogram_from(r["key"][~same], r["q"][~same], r["cls"][~same], tiny.sc.n_bins)
    np.testing.assert_array_equal(acc - gm, rm)
    assert np.all(acc % (1 << 32) == 0)


def test_result_independent_of_launch_shape_and_partition(tiny):
    n = 150_001
    ref = None
    for block, grid in [(512, 0), (256, 0), (64, 7), (128, 1000), (256, 3), (32, 152 * 40)]:
        tiny.zero()
        tiny.run(SEED + 2, 5, n, listmode=False, block=block, grid=grid)
        a = tiny.acc()
        if ref is None:
            ref = a.clone()
        else:
            assert bool((a == ref).all()), f"block {block} grid {grid} differs"
    tiny.zero()
    for lo, hi in [(5, 40_000), (40_000, 40_001), (40_001, n + 5)]:
        tiny.run(SEED + 2, lo, hi - lo, listmode=False)
    assert bool((tiny.acc() == ref).all())


_FIRST_LAUNCH = '''
import json, sys
sys.path.insert(0, "tests")
import workloads as W
from gpu_helpers import Session
sc = W.scanner_tiny()
s = Session(sc, W.standard_materials(), W.phantom_water_cylinder(), W.lut_tiny(sc))
a = s.run(1, 0, 2_000_000, listmode=False)["stats"]
b = s.run(1, 0, 2_000_000, listmode=False)["stats"]
print(json.dumps([a["grid"], a["block"], b["grid"], b["block"]]))
s.close()
'''


def test_first_launch_of_a_process_fills_every_sm_twice():
    """The automatic launch shape is 512-thread CTAs, two per SM, from the
    first launch of a fresh process on (the occupancy query counts the
    kernel's dynamic shared memory only once the kernel may use it)."""
    import json
    import os
    import subprocess
    import sys
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.check_output([sys.executable, "-c", _FIRST_LAUNCH], cwd=root, text=True, timeout=600)
    g1, b1, g2, b2 = json.loads(out.strip().splitlines()[-1])
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert (g1, b1) == (g2, b2) == (2 * sms, 512)


def test_checkpoint_resume_is_bit_identical(tiny):
    import torch
    n = 120_000
    tiny.zero()
    tiny.run(SEED + 3, 0, n, listmode=False)
    full = tiny.acc()
    tiny.zero()
    tiny.run(SEED + 3, 0, n // 3, listmode=False)
    ck = tiny.acc()                                   # checkpoint: (seed, next id, acc)
    acc2 = psc.psc_acc_create(tiny.ctx, tiny.s_id)
    psc.psc_acc_write(tiny.ctx, acc2, ck, tiny.stream())
    tiny.run(SEED + 3, n // 3, n - n // 3, listmode=False, acc=acc2)
    assert bool((tiny.acc(acc2) == full).all())
    psc.psc_unload(tiny.ctx, acc2)
    torch.cuda.synchronize()


@pytest.mark.parametrize("dtype,bound", [(psc.PSC_LUT_F16, 2e-3), (psc.PSC_LUT_BF16, 1.6e-2)])
def test_reduced_precision_lut_error_is_bounded(tiny, dtype, bound):
    """FP16/BF16 LUT storage: the weight error against the FP64 oracle is
    bounded by the storage rounding (2^-11 / 2^-8 relative per tap)."""
    l_id = psc.psc_load_lut(tiny.ctx, psc.lut_desc(tiny.lut, dtype).desc)
    n = 200_000
    tiny.zero()
    g = tiny.run(SEED, 0, n, lut=l_id)
    r = oracle.simulate(tiny.sc, tiny.mats, tiny.ph, tiny.lut, SEED, 0, n, threads=8)
    same = compare_histories(g, r, w_rtol=bound)
    det = same & (r["key"] >= 0)
    rel = np.abs(g["q"][det] - r["q"][det]) / r["q"][det]
    print(f"LUT dtype {dtype}: max weight rel err {rel.max():.3g}, mean {rel.mean():.3g}")
    psc.psc_unload(tiny.ctx, l_id)


def test_vacuum_trues_geometry(tiny):
    """mu = 0: all pairs fly straight; binned trues match the oracle."""
    ph = W.phantom_uniform_box(dims=(20, 20, 10), voxel=(5.0, 5.0, 5.0), material=W.MAT_VACUUM,
                               density=0.0, source="uniform")
    p_id = psc.psc_load_phantom(tiny.ctx, psc.phantom_desc(ph).desc, tiny.m_id)
    n = 100_000
    tiny.zero()
    g = tiny.run(7, 0, n, phantom=p_id, bin_mask=3)
    r = oracle.simulate(tiny.sc, tiny.mats, ph, tiny.lut, 7, 0, n, threads=8, bin_mask=3)
    compare_histories(g, r)
    assert (g["cls"] == 7).sum() == 0 and (g["cls"] == 6).sum() > 1000
    psc.psc_unload(tiny.ctx, p_id)


def test_update_activity_rebuilds_emission(tiny):
    rng = np.random.default_rng(0)
    act = (tiny.ph.activity * rng.uniform(0.0, 2.0, tiny.ph.activity.shape)).astype(np.float32)
    psc.psc_update_activity(tiny.ctx, tiny.p_id, act)
    ph2 = W.Phantom(tiny.ph.dims, tiny.ph.voxel, tiny.ph.origin, tiny.ph.material,
                    tiny.ph.density, act)
    n = 100_000
    tiny.zero()
    g = tiny.run(SEED, 0, n)
    r = oracle.simulate(tiny.sc, tiny.mats, ph2, tiny.lut, SEED, 0, n, threads=8)
    compare_histories(g, r)
    psc.psc_update_activity(tiny.ctx, tiny.p_id, tiny.ph.activity)


def test_edge_cases(tiny):
    tiny.zero()
    g = tiny.run(SEED, 0, 0)                               # empty range: no work, zeros
    assert sum(g["stats"][c] for c in psc.CLASSES) == 0
    assert int(tiny.acc().abs().sum()) == 0
    g = tiny.run(SEED, 2**64 - 2, 1)                       # one history at the top of the id range
    r = oracle.simulate(tiny.sc, tiny.mats, tiny.ph, tiny.lut, SEED, 2**64 - 2, 1)
    assert g["cls"][0] == r["cls"][0] and g["key"][0] == r["key"][0]
    with pytest.raises(psc.PscError) as e:
        tiny.run(SEED, 2**64 - 1, 2)
    assert e.value.code == psc.PSC_EOVERFLOW
    with pytest.raises(psc.PscError) as e:
        tiny.run(SEED, 0, 10, phantom=999)
    assert e.value.code == psc.PSC_ENOTFOUND
    with pytest.raises(psc.PscError) as e:
        tiny.run(SEED, 0, 10, acc=tiny.l_id)                 # wrong object kind
    assert e.value.code == psc.PSC_ENOTFOUND
    for block in (100, 1024):
        with pytest.raises(psc.PscError) as e:
            tiny.run(SEED, 0, 10, block=block)
        assert e.value.code == psc.PSC_EINVAL
    bad = W.phantom_water_cylinder()
    bad.activity[:] = 0
    with pytest.raises(psc.PscError) as e:
        psc.psc_load_phantom(tiny.ctx, psc.phantom_desc(bad).desc, tiny.m_id)
    assert e.value.code == psc.PSC_EINVAL
    big = W.phantom_uniform_box(dims=(200, 200, 4), voxel=(4.0, 4.0, 4.0))   # 800 mm wide
    p_id = psc.psc_load_phantom(tiny.ctx, psc.phantom_desc(big).desc, tiny.m_id)
    with pytest.raises(psc.PscError) as e:
        tiny.run(SEED, 0, 10, phantom=p_id)
    assert e.value.code == psc.PSC_EINVAL and "cylinder" in str(e.value)
    psc.psc_unload(tiny.ctx, p_id)
    wrong = W.lut_smooth(4, 4, 4, 3, 3, 425.0)
    l_id = psc.psc_load_lut(tiny.ctx, psc.lut_desc(wrong).desc)
    with pytest.raises(psc.PscError) as e:
        tiny.run(SEED, 0, 10, lut=l_id)
    assert e.value.code == psc.PSC_EINVAL
    psc.psc_unload(tiny.ctx, l_id)
    out_of_range = W.lut_tiny(tiny.sc)
    out_of_range.data[0, 0, 0, 0, 0] = 1.5
    with pytest.raises(psc.PscError):
        psc.psc_load_lut(tiny.ctx, psc.lut_desc(out_of_range).desc)


def test_independent_seeds_pass_per_bin_poisson_chi_square(tiny):
    """Independent seeds on the GPU give count sinograms (LUT = 1) whose
    every bin holds Poisson counts of one mean: the per-bin two-sample test
    of tests/poisson.py over the 137.5 M-bin tiny sinogram at 2e8 histories
    per seed (mostly 0-3 counts per bin, where the exact-moment form
    decides)."""
    from poisson import assert_same_poisson_means
    out = []
    for seed in (101, 202):
        tiny.zero()
        tiny.run(seed, 0, 200_000_000, listmode=False, lut=0, stats=False)
        out.append(tiny.acc().cpu().numpy() >> 32)
    res = assert_same_poisson_means(*out)
    assert res["bins"] > 500_000


def test_gpu_and_oracle_sinograms_have_the_same_per_bin_means():
    """The GPU's count sinogram and the oracle's, from different seeds, are
    draws of one per-bin Poisson distribution (small scanner, tens of counts
    per bin): the kernel samples the oracle's process, not only itself."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from poisson import assert_same_poisson_means
    sc = W.scanner_small(n_crystals=16, n_rings=4, n_tof=5, ring_pitch=40.0, e_lo=350.0)
    ph = W.phantom_water_cylinder(dims=(32, 32, 16), voxel=(4.0, 4.0, 4.0), radius=60.0)
    mats = W.standard_materials()
    n = 4_000_000
    s = Session(sc, mats, ph, None)
    try:
        s.zero()
        s.run(SEED + 71, 0, n, listmode=False, lut=0, stats=False)
        g = s.acc().cpu().numpy() >> 32
    finally:
        s.close()
    r = oracle.simulate(sc, mats, ph, None, SEED + 72, 0, n, threads=8)
    m = r["cls"] == oracle.SCATTER
    res = assert_same_poisson_means(g, np.bincount(r["key"][m], minlength=sc.n_bins))
    assert res["mean_count"] > 20


# --------------------------------------------------------------------------
# paper-scale configuration (full-size phantom, scanner, LUT; sampled
# history ranges compared one by one with the oracle)
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def signa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_signa()
    mats = W.standard_materials()
    ph = W.phantom_torso()
    lut = W.lut_signa(sc)
    s = Session(sc, mats, ph, lut)
    s.mats, s.ph, s.lut = mats, ph, lut
    yield s
    s.close()


@pytest.mark.parametrize("first,n", [(0, 100_000), (500_000_017, 60_001)])
def test_signa_histories_match_oracle(signa, first, n):
    g = signa.run(SEED, first, n)
    r = oracle.simulate(signa.sc, signa.mats, signa.ph, signa.lut, SEED, first, n, threads=8)
    compare_histories(g, r)
    assert (r["cls"] == 7).sum() > 0.02 * n


def test_signa_large_launch_properties(signa):
    """1e8 histories in the benchmark's launch configuration: class counts
    add up, the accumulator total equals the binned weight sum, and the
    last histories of the range match the oracle one by one."""
    import torch
    n = 100_000_000
    signa.zero()
    st = signa.run(SEED, 0, n, listmode=False)["stats"]
    assert sum(st[c] for c in psc.CLASSES) == n
    acc = signa.acc()
    assert int(acc.sum()) == st["weight_sum"]
    assert int((acc > 0).sum()) <= st["binned"]
    del acc
    signa.zero()
    tail = signa.run(SEED, n - 20_000, 20_000)
    r = oracle.simulate(signa.sc, signa.mats, signa.ph, signa.lut, SEED, n - 20_000, 20_000, threads=8)
    compare_histories(tail, r)
    torch.cuda.synchronize()


def test_alias_table_equals_oracle(tiny):
    """The runtime's alias table (thresholds on the Philox word) makes the
    same accept decision as the oracle's FP64 Vose table for every voxel."""
    rng = np.random.default_rng(3)
    act = (tiny.ph.activity * rng.exponential(size=tiny.ph.activity.shape)).astype(np.float32)
    psc.psc_update_activity(tiny.ctx, tiny.p_id, act)
    thr, alias = psc.psc_phantom_alias(tiny.ctx, tiny.p_id, act.size)
    prob, oalias = oracle.alias_build(act)
    np.testing.assert_array_equal(alias, oalias)
    # k < thr  <=>  (2k + 1) 2^-24 < prob, checked at the boundary and at random k
    for k in (thr.astype(np.int64) - 1, thr.astype(np.int64), rng.integers(0, 1 << 23, act.size)):
        k = np.clip(k, 0, (1 << 23) - 1)
        np.testing.assert_array_equal(k < thr, (2 * k + 1) * 2.0**-24 < prob)
    psc.psc_update_activity(tiny.ctx, tiny.p_id, tiny.ph.activity)


def test_energy_resolution_variant_matches_oracle():
    """No-LUT mode of Sec. 2.2.1: 11.2 % energy resolution and a 425-650 keV
    window.  The blurred energy decides the window on both sides from the
    same two words of the photon's stream, so histories match as without
    resolution; some photons below 425 keV are detected."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_tiny()
    sc.e_res = 0.112
    mats, ph = W.standard_materials(), W.phantom_water_cylinder()
    s = Session(sc, mats, ph, None)
    try:
        n = 200_000
        g = s.run(SEED + 21, 0, n, lut=0)
        r = oracle.simulate(sc, mats, ph, None, SEED + 21, 0, n, threads=8, records=True)
        same = compare_histories(g, r)
        assert (~same).sum() <= 0.001 * n
        rec = r["rec"]
        det = rec["status"] == oracle.DETECTED
        assert np.any(det & (rec["energy"] < sc.e_lo))
        # the window's decisions differ from those on exact energies at the same seed
        exact = oracle.simulate(W.scanner_tiny(), mats, ph, None, SEED + 21, 0, n, threads=8)
        assert (g["cls"] == oracle.ENERGY_WINDOW).sum() != (exact["cls"] == oracle.ENERGY_WINDOW).sum()
    finally:
        s.close()


def _vacuum_box():
    return W.phantom_uniform_box(dims=(32, 32, 24), voxel=(4.0, 4.0, 4.0), material=W.MAT_VACUUM, density=0.0)


@pytest.mark.parametrize("mode,phantom", [(1, "vacuum"), (2, "vacuum"), (2, "torso")])
def test_gap_model_matches_oracle(mode, phantom):
    """Gaps between the 28 modules and 5 blocks of the paper-scale scanner
    (Sec. 2.2.1-2.2.2).  Mode 1 loses photons in a gap; mode 2 weights them
    with the LUT value of their virtual crystal and assigns them to an edge
    crystal from one word of the photon's stream per gap.  Histories match
    the oracle's one by one, and the sampled histories reach the gaps."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_signa_gaps(gap_mode=mode)
    mats = W.standard_materials()
    ph = _vacuum_box() if phantom == "vacuum" else W.phantom_torso()
    lut = W.lut_signa(sc)
    s = Session(sc, mats, ph, lut)
    try:
        n = 100_000
        g = s.run(SEED + 31, 0, n)
        r = oracle.simulate(sc, mats, ph, lut, SEED + 31, 0, n, threads=8, records=True)
        same = compare_histories(g, r)
        assert (~same).sum() <= 0.001 * n
        rec = r["rec"]
        det = np.flatnonzero((rec["status"] == oracle.DETECTED).any(axis=1))[:4000]
        in_gap = sum(oracle.place(sc, rec["hit"][i, k])[0] != 0
                     for i in det for k in range(2) if rec["status"][i, k] == oracle.DETECTED)
        if mode == 1:
            assert in_gap == 0 and (g["cls"] == oracle.LOST_AXIAL).sum() > 0.05 * n
        else:
            assert in_gap > 100
            # histories with a photon in a gap are binned and match
            gap_rows = [i for i in det if (rec["status"][i] == oracle.DETECTED).all()
                        and any(oracle.place(sc, rec["hit"][i, k])[0] for k in range(2))]
            gap_rows = np.array(gap_rows)
            assert same[gap_rows].mean() >= 0.99
    finally:
        s.close()


def test_gap_scanner_rejects_a_lut_without_virtual_crystals():
    """The LUT of a scanner with gaps has module_t + 2 transaxial and
    n_blocks (module_a + 2) axial positions; a gapless LUT is refused."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_signa_gaps(gap_mode=2)
    plain = W.scanner_signa()
    s = Session(sc, W.standard_materials(), _vacuum_box(), W.lut_signa(plain))
    try:
        with pytest.raises(psc.PscError) as e:
            s.run(SEED, 0, 1000)
        assert e.value.code == psc.PSC_EINVAL
    finally:
        s.close()


@pytest.mark.parametrize("keep,gaps", [(("e",), 0), (("e", "a", "b"), 0), (("e", "t", "z"), 0),
                                       (("e", "a", "b"), 1), (("e", "t", "z"), 2)])
def test_lower_dimensional_luts_match_oracle(keep, gaps):
    """Sec. 2.2.2's lower-dimensional LUTs, made by summing synthetic
    histograms over the dropped axes: energy only, energy and angles, energy
    and crystals; the paper pairs the LUTs without crystal information with
    dropping gap photons and the energy-and-crystal LUT with edge-crystal
    assignment.  Per-history parity with the oracle."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if gaps:
        sc, ph, n = W.scanner_signa_gaps(gap_mode=gaps), W.phantom_torso(), 100_000
        full = W.lut_signa(sc)
    else:
        sc, ph, n = W.scanner_tiny(), W.phantom_water_cylinder(), 200_000
        full = W.lut_tiny(sc)
    inc, det = W.lut_histograms(full, counts=50.0)
    lut = W.lut_reduced(full, inc, det, keep)
    mats = W.standard_materials()
    s = Session(sc, mats, ph, lut)
    try:
        g = s.run(SEED + 41, 0, n)
        r = oracle.simulate(sc, mats, ph, lut, SEED + 41, 0, n, threads=8)
        same = compare_histories(g, r)
        assert (~same).sum() <= 0.001 * n
        assert (r["cls"] == 7).sum() > 0.001 * n
    finally:
        s.close()


def test_listmode_records_match_oracle(tiny):
    """The listmode debug output (Sec. 2.2.1: the simulator's list of
    coincidences): one record per history whose photons are both detected
    in different crystals, holding the emission voxel, the exact energies,
    the cylindrical hit coordinates, the directions, the scatter counts and
    Rayleigh flags, and the crystals of the oracle's record of the same
    history; the records' weights and classes are those of the per-history
    outputs."""
    import torch
    n, cap = 150_000, 150_000
    dev = torch.device("cuda:0")
    dt = psc.listmode_dtype()
    lm = torch.zeros(cap * dt.itemsize, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    cls = torch.full((n,), -1, dtype=torch.int8, device=dev)
    q = torch.full((n,), -2, dtype=torch.int64, device=dev)
    key = torch.full((n,), -2, dtype=torch.int64, device=dev)
    tiny.zero()
    args = psc.sim_args(SEED + 51, 0, n, tiny.s_id, tiny.p_id, tiny.a_id, lut=tiny.l_id,
                        bin_mask=psc.PSC_BIN_SCATTER | psc.PSC_BIN_TRUES, cls_out=cls, key_out=key,
                        q_out=q, lm_out=lm, lm_count=cnt, lm_capacity=cap)
    psc.psc_simulate(tiny.ctx, args, stream=tiny.stream())
    torch.cuda.synchronize()
    g_cls, g_q, m = cls.cpu().numpy(), q.cpu().numpy(), int(cnt.item())
    rec = np.frombuffer(lm[: m * dt.itemsize].cpu().numpy().tobytes(), dtype=dt)
    rec = rec[np.argsort(rec["history"])]
    coinc = np.flatnonzero(np.isin(g_cls, [5, 6, 7]))
    assert m == coinc.size > 1000
    np.testing.assert_array_equal(rec["history"], coinc)
    np.testing.assert_array_equal(rec["cls"], g_cls[coinc])
    in_range = rec["cls"] != 5
    np.testing.assert_array_equal(rec["q"][in_range], g_q[coinc][in_range])
    assert (rec["pad"] == 0).all()
    r = oracle.simulate(tiny.sc, tiny.mats, tiny.ph, tiny.lut, SEED + 51, 0, n, threads=8, records=True)["rec"]
    o = r[coinc]
    same = (o["cls"] == rec["cls"]) & (o["key"] == key.cpu().numpy()[coinc])
    assert same.mean() > 0.999
    o, g = o[same], rec[same]
    np.testing.assert_array_equal(g["voxel"], o["voxel"])
    np.testing.assert_array_equal(g["crystal"], o["crystal"])
    np.testing.assert_array_equal(g["ring"], o["ring"])
    np.testing.assert_array_equal(g["n_scatter"], o["n_compton"] + o["n_rayleigh"])
    np.testing.assert_array_equal(g["rayleigh"], (o["n_rayleigh"] > 0).astype(np.uint8))
    np.testing.assert_allclose(g["energy_kev"], o["energy"], rtol=2e-5)
    np.testing.assert_allclose(g["dir"], o["exit_dir"], atol=2e-5)
    phi = np.mod(np.arctan2(o["hit"][..., 1], o["hit"][..., 0]), 2 * np.pi)
    dphi = np.abs(g["phi"] - phi)
    assert np.minimum(dphi, 2 * np.pi - dphi).max() < 1e-4
    np.testing.assert_allclose(g["z_mm"], o["hit"][..., 2], atol=2e-3)
    np.testing.assert_allclose(g["delta_mm"], 0.5 * (o["path"][:, 0] - o["path"][:, 1]), atol=5e-3)
    assert (g["n_scatter"] > 0).any() and (g["n_scatter"] == 0).any()


def test_listmode_capacity_counts_beyond_the_buffer(tiny):
    """Records past lm_capacity are counted but not written; lm_out needs
    lm_count."""
    import torch
    dev = torch.device("cuda:0")
    dt = psc.listmode_dtype()
    cap = 10
    lm = torch.full(((cap + 1) * dt.itemsize,), 0xAB, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    args = psc.sim_args(SEED + 52, 0, 50_000, tiny.s_id, tiny.p_id, tiny.a_id, lut=tiny.l_id,
                        lm_out=lm, lm_count=cnt, lm_capacity=cap)
    psc.psc_simulate(tiny.ctx, args, stream=tiny.stream())
    torch.cuda.synchronize()
    assert int(cnt.item()) > cap
    tail = lm[cap * dt.itemsize:].cpu().numpy()
    assert (tail == 0xAB).all()  # the record after the capacity is untouched
    bad = psc.sim_args(SEED, 0, 10, tiny.s_id, tiny.p_id, tiny.a_id, lm_out=lm, lm_capacity=cap)
    with pytest.raises(psc.PscError) as e:
        psc.psc_simulate(tiny.ctx, bad, stream=tiny.stream())
    assert e.value.code == psc.PSC_EINVAL


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16", "none"])
def test_production_kernel_equals_debug_kernel(tiny, dtype):
    """The production instantiations (no counters, no listmode; a single f32
    job reads its parameters from the kernel parameters) add exactly the
    accumulator of the instantiation the parity tests check."""
    dts = {"f32": psc.PSC_LUT_F32, "f16": psc.PSC_LUT_F16, "bf16": psc.PSC_LUT_BF16}
    lut = psc.psc_load_lut(tiny.ctx, psc.lut_desc(tiny.lut, dts[dtype]).desc) if dtype in dts else 0
    n = 300_000
    tiny.zero()
    tiny.run(SEED + 61, 0, n, listmode=False, lut=lut, stats=True)
    debug = tiny.acc().clone()
    tiny.zero()
    tiny.run(SEED + 61, 0, n, listmode=False, lut=lut, stats=False)
    prod = tiny.acc()
    assert int(debug.sum()) > 0
    assert bool((prod == debug).all())
    if lut:
        psc.psc_unload(tiny.ctx, lut)


# --------------------------------------------------------------------------
# the TOF blur path of the production kernel
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny_blur():
    """The tiny configuration with a Gaussian TOF blur (sigma 20 mm on 13
    bins of 50 mm), so the coincidence section reads stream 0, block 2."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = W.scanner_tiny()
    sc.tof_sigma_mm = 20.0
    mats, ph, lut = W.standard_materials(), W.phantom_water_cylinder(), W.lut_tiny(sc)
    s = Session(sc, mats, ph, lut)
    s.mats, s.ph, s.lut = mats, ph, lut
    yield s
    s.close()


def test_blurred_tof_histories_match_oracle(tiny_blur):
    n = 200_000
    tiny_blur.zero()
    g = tiny_blur.run(SEED + 81, 0, n)
    r = oracle.simulate(tiny_blur.sc, tiny_blur.mats, tiny_blur.ph, tiny_blur.lut, SEED + 81, 0, n, threads=8)
    same = compare_histories(g, r)
    # the blur moves events across TOF bins: the unblurred run bins differently
    plain = oracle.simulate(W.scanner_tiny(), tiny_blur.mats, tiny_blur.ph, tiny_blur.lut, SEED + 81, 0, n,
                            threads=8)
    det = same & (r["key"] >= 0)
    assert np.mean(r["key"][det] != plain["key"][det]) > 0.2


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16", "none"])
def test_production_kernel_with_tof_blur_equals_debug_kernel(tiny_blur, dtype):
    """The production instantiations on the blur path (for f32: the
    single-job, parameter-operand, 512-thread kernel the benchmark times)
    add exactly the accumulator of the debug instantiation that the
    per-history parity tests check against the oracle."""
    dts = {"f32": psc.PSC_LUT_F32, "f16": psc.PSC_LUT_F16, "bf16": psc.PSC_LUT_BF16}
    s = tiny_blur
    lut = psc.psc_load_lut(s.ctx, psc.lut_desc(s.lut, dts[dtype]).desc) if dtype in dts else 0
    n = 400_000
    s.zero()
    s.run(SEED + 62, 0, n, listmode=False, lut=lut, stats=True)
    debug = s.acc().clone()
    s.zero()
    s.run(SEED + 62, 0, n, listmode=False, lut=lut, stats=False)
    prod = s.acc()
    assert int(debug.sum()) > 0
    assert bool((prod == debug).all())
    if lut:
        psc.psc_unload(s.ctx, lut)


def _nonzero(t):
    import torch
    idx = torch.nonzero(t).squeeze(1)
    return idx.cpu().numpy(), t[idx].cpu().numpy()


def test_signa_production_kernel_equals_debug_kernel(signa):
    """The benchmark's exact kernel (single f32 job, 512-thread CTAs, the
    400 ps TOF blur) on the paper-scale configuration adds the same
    accumulator, bin for bin, as the debug instantiation that the paper-scale
    per-history tests compare with the oracle."""
    n = 3_000_000
    signa.zero()
    signa.run(SEED + 63, 7, n, listmode=False, stats=True)
    t = signa.acc()
    d_idx, d_val = _nonzero(t)
    del t
    signa.zero()
    signa.run(SEED + 63, 7, n, listmode=False, stats=False)
    t = signa.acc()
    p_idx, p_val = _nonzero(t)
    del t
    assert d_idx.size > 50_000
    np.testing.assert_array_equal(p_idx, d_idx)
    np.testing.assert_array_equal(p_val, d_val)
