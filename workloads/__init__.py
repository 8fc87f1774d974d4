"""Seeded synthetic inputs for the PET scatter Monte Carlo path.

This module builds the *inputs* of a scatter simulation: scanner geometry,
material cross-section tables, voxel phantoms (material, density, activity),
the 5D single-photon detection-probability LUT, and sensitivity /
normalisation sinograms.  It is imported by the tests, by the benchmark and
by the oracle's tests alike.  It contains none of the simulation method's
arithmetic (no sampling, transport, detection, weighting, binning or
smoothing): only the construction of the data those steps consume.

Units: lengths in mm, energies in keV, densities in g/cm^3, mass attenuation
coefficients in cm^2/g, angles in degrees.

Arrays are numpy; voxel arrays are laid out [nz][ny][nx] (x fastest), the
LUT [apos][tpos][E][alpha][beta] (beta fastest), sinograms
[plane][view][radial][tof] (tof fastest) or, for per-LOR (non-TOF) inputs,
[plane][view][radial].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Physical constants (CODATA 2018)
# ---------------------------------------------------------------------------
ELECTRON_REST_KEV = 511.0  # the path uses E' = E / (1 + (E/511)(1 - cos)) with 511 keV
CLASSICAL_ELECTRON_RADIUS_CM = 2.8179403262e-13
AVOGADRO = 6.02214076e23
SPEED_OF_LIGHT_MM_PER_PS = 0.299792458

N_ENERGY_NODES = 513  # table nodes at E = 0, 1, ..., 512 keV

# material ids used by the synthetic phantoms
MAT_VACUUM, MAT_WATER, MAT_LUNG, MAT_BONE = 0, 1, 2, 3


# ---------------------------------------------------------------------------
# Cross-section tables (project-chosen analytic physics; the paper uses the
# simulator's own material files and does not state them)
# ---------------------------------------------------------------------------
def klein_nishina_sigma_cm2(e_kev):
    """Total Klein-Nishina cross section per free electron (cm^2).

    Closed form of the integral of the Klein-Nishina differential cross
    section over the full solid angle (Klein & Nishina 1929; e.g. Evans,
    "The Atomic Nucleus", ch. 23).
    """
    a = np.asarray(e_kev, dtype=np.float64) / ELECTRON_REST_KEV
    l = np.log1p(2.0 * a)
    t1 = (1.0 + a) / a**2 * (2.0 * (1.0 + a) / (1.0 + 2.0 * a) - l / a)
    t2 = l / (2.0 * a)
    t3 = (1.0 + 3.0 * a) / (1.0 + 2.0 * a) ** 2
    return 2.0 * math.pi * CLASSICAL_ELECTRON_RADIUS_CM**2 * (t1 + t2 - t3)


@dataclass
class Material:
    """One material: mass attenuation tables on the 1 keV grid + Rayleigh
    form-factor parameter kappa (see ``rayleigh`` notes in the oracle)."""
    name: str
    compton: np.ndarray      # f64[513] cm^2/g
    rayleigh: np.ndarray     # f64[513] cm^2/g
    photo: np.ndarray        # f64[513] cm^2/g
    kappa: float             # Rayleigh form factor width parameter (dimensionless)


def make_material(name, z_over_a, k_photo, r_rayl, kappa, vacuum=False):
    """Analytic tables: Compton = (Z/A) N_A sigma_KN(E); photoelectric =
    k_photo (E/100 keV)^-3; Rayleigh = r_rayl (E/100 keV)^-2.  Values at
    E < 1 keV are held at their 1 keV value (only E >= the energy window
    matters to the simulation)."""
    e = np.maximum(np.arange(N_ENERGY_NODES, dtype=np.float64), 1.0)
    if vacuum:
        z = np.zeros(N_ENERGY_NODES)
        return Material(name, z.copy(), z.copy(), z.copy(), 0.0)
    compton = z_over_a * AVOGADRO * klein_nishina_sigma_cm2(e)
    photo = k_photo * (e / 100.0) ** -3
    rayl = r_rayl * (e / 100.0) ** -2
    return Material(name, compton, rayl, photo, float(kappa))


def standard_materials():
    """[vacuum, water, lung, bone].  Lung is water composition (its 0.3 g/cc
    density lives in the phantom); bone is cortical-like (Z/A 0.5148) with a
    larger photoelectric and Rayleigh strength."""
    return [
        make_material("vacuum", 0, 0, 0, 0, vacuum=True),
        make_material("water", 10.0 / 18.01528, 2.76e-3, 2.76e-3, 500.0),
        make_material("lung", 10.0 / 18.01528, 2.76e-3, 2.76e-3, 500.0),
        make_material("bone", 0.5148, 1.9e-2, 5.0e-3, 800.0),
    ]


def materials_arrays(mats):
    """Stack a material list into contiguous arrays (n_mat, 513) + kappa."""
    comp = np.ascontiguousarray(np.stack([m.compton for m in mats]), dtype=np.float64)
    rayl = np.ascontiguousarray(np.stack([m.rayleigh for m in mats]), dtype=np.float64)
    phot = np.ascontiguousarray(np.stack([m.photo for m in mats]), dtype=np.float64)
    kap = np.ascontiguousarray([m.kappa for m in mats], dtype=np.float64)
    return comp, rayl, phot, kap


# ---------------------------------------------------------------------------
# Scanner geometry
# ---------------------------------------------------------------------------
@dataclass
class Scanner:
    radius: float          # mm, cylinder at the depth of interaction
    n_crystals: int        # crystals per ring (even)
    n_rings: int
    ring_pitch: float      # mm; axial extent L = n_rings * ring_pitch, centred on z=0
    module_t: int          # crystals per module transaxially (LUT tpos = c mod module_t)
    module_a: int          # rings per block axially (LUT apos = ring mod module_a)
    e_lo: float            # keV energy window
    e_hi: float
    n_tof: int
    tof_bin_mm: float      # TOF bin width in half-path-difference units (mm)
    tof_sigma_mm: float    # Gaussian TOF blur sigma (mm), 0 = none
    n_rad: int = 0         # radial bins kept (centred clip); 0 -> n_crystals - 1
    e_res: float = 0.0     # energy resolution FWHM / 511 keV at 511 keV (scaling as sqrt(E)); 0 = exact
    gap_mode: int = 0      # 0 no gaps; 1 photons in gaps are lost; 2 they go to an edge crystal
    gap_t: float = 0.0     # transaxial gap between modules (mm at the detection radius)
    gap_a: float = 0.0     # axial gap between blocks (mm)
    crystal_depth: float = 25.0   # mm (a project choice: the paper gives no block geometry)
    doi: float = 7.0       # depth of the detection cylinder below the block face (mm, project choice)
    mu_block: float = 0.0869      # LYSO attenuation at 511 keV (1/mm)

    def __post_init__(self):
        if self.n_rad == 0:
            self.n_rad = self.n_crystals - 1

    @property
    def length(self):
        return self.n_rings * self.ring_pitch

    @property
    def n_planes(self):
        return self.n_rings * self.n_rings

    @property
    def n_views(self):
        return self.n_crystals // 2

    @property
    def shape(self):
        return (self.n_planes, self.n_views, self.n_rad, self.n_tof)

    @property
    def n_tpos(self):
        """LUT transaxial positions: module-local crystals (+ 2 virtual with gaps)."""
        return self.module_t + 2 if self.gap_mode else self.module_t

    @property
    def n_apos(self):
        """LUT axial positions: block-local rings, or every block's rings + 2 virtual with gaps."""
        return (self.n_rings // self.module_a) * (self.module_a + 2) if self.gap_mode else self.module_a

    @property
    def n_bins(self):
        return self.n_planes * self.n_views * self.n_rad * self.n_tof

    @property
    def lor_shape(self):
        return (self.n_planes, self.n_views, self.n_rad)


def tof_sigma_from_fwhm_ps(fwhm_ps):
    """sigma of the half path difference (l_a - l_b)/2 for a coincidence
    timing FWHM in ps: dx = c dt / 2."""
    return SPEED_OF_LIGHT_MM_PER_PS * fwhm_ps / 2.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))


def scanner_tiny():
    """Tiny configuration: R = 310 mm, 288 crystals x 16 rings of 4 mm,
    425-650 keV, 13 TOF bins of 50 mm, no TOF blur."""
    return Scanner(radius=310.0, n_crystals=288, n_rings=16, ring_pitch=4.0,
                   module_t=4, module_a=4, e_lo=425.0, e_hi=650.0,
                   n_tof=13, tof_bin_mm=50.0, tof_sigma_mm=0.0)


def scanner_signa():
    """Paper-scale configuration shaped like the Signa PET/MR (Sec. 2.1.1):
    448 crystals/ring (28 modules x 16), 45 rings (5 blocks x 9), axial length
    250.4 mm, radius 311.8 mm taken at the depth of interaction; window
    300-650 keV (the LUT setting of Sec. 2.2.1); 27 TOF bins of 24 mm with a
    400 ps FWHM Gaussian TOF blur."""
    return Scanner(radius=311.8, n_crystals=448, n_rings=45, ring_pitch=250.4 / 45,
                   module_t=16, module_a=9, e_lo=300.0, e_hi=650.0,
                   n_tof=27, tof_bin_mm=24.0, tof_sigma_mm=tof_sigma_from_fwhm_ps(400.0))


def scanner_signa_gaps(gap_mode=2, gap_t=2.0, gap_a=2.0):
    """The paper-scale scanner with gaps between its 28 modules and 5 axial
    blocks (Sec. 2.2.1-2.2.2; the LUT then has 18 x 55 positions).  The gap
    widths, crystal depth and depth of interaction are project choices: the
    paper gives no block geometry."""
    sc = scanner_signa()
    sc.gap_mode, sc.gap_t, sc.gap_a = gap_mode, gap_t, gap_a
    return sc


def scanner_small(n_crystals=16, n_rings=4, n_tof=5, radius=120.0, ring_pitch=8.0,
                  tof_bin_mm=40.0, tof_sigma_mm=0.0, e_lo=425.0, e_hi=650.0,
                  module_t=4, module_a=2, n_rad=0):
    """Small scanner for brute-force tests."""
    return Scanner(radius=radius, n_crystals=n_crystals, n_rings=n_rings,
                   ring_pitch=ring_pitch, module_t=module_t, module_a=module_a,
                   e_lo=e_lo, e_hi=e_hi, n_tof=n_tof, tof_bin_mm=tof_bin_mm,
                   tof_sigma_mm=tof_sigma_mm, n_rad=n_rad)


# ---------------------------------------------------------------------------
# Phantoms
# ---------------------------------------------------------------------------
@dataclass
class Phantom:
    dims: tuple            # (nx, ny, nz)
    voxel: tuple           # (dx, dy, dz) mm
    origin: tuple          # (ox, oy, oz) mm: min corner of voxel (0,0,0)
    material: np.ndarray   # u8[nz, ny, nx]
    density: np.ndarray    # f32[nz, ny, nx]
    activity: np.ndarray   # f32[nz, ny, nx]

    @property
    def n_voxels(self):
        return int(np.prod(self.dims))


def _centres(dims, voxel):
    nx, ny, nz = dims
    dx, dy, dz = voxel
    x = (np.arange(nx) + 0.5 - nx / 2.0) * dx
    y = (np.arange(ny) + 0.5 - ny / 2.0) * dy
    z = (np.arange(nz) + 0.5 - nz / 2.0) * dz
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    return xx, yy, zz


def _centred_origin(dims, voxel):
    return tuple(-0.5 * n * d for n, d in zip(dims, voxel))


def _finish(dims, voxel, mat, dens, act):
    return Phantom(tuple(int(v) for v in dims), tuple(float(v) for v in voxel),
                   _centred_origin(dims, voxel),
                   np.ascontiguousarray(mat, dtype=np.uint8),
                   np.ascontiguousarray(dens, dtype=np.float32),
                   np.ascontiguousarray(act, dtype=np.float32))


def phantom_water_cylinder(dims=(64, 64, 32), voxel=(4.0, 4.0, 4.0), radius=100.0,
                           half_length=100.0, activity=1.0):
    """Uniform water cylinder (axis z, centred) with uniform activity; voxels
    whose centre lies outside are vacuum with zero activity.  The cylinder is
    clipped to the grid where it is longer."""
    xx, yy, zz = _centres(dims, voxel)
    inside = (xx**2 + yy**2 <= radius**2) & (np.abs(zz) <= half_length)
    mat = np.where(inside, MAT_WATER, MAT_VACUUM)
    dens = np.where(inside, 1.0, 0.0)
    act = np.where(inside, activity, 0.0)
    return _finish(dims, voxel, mat, dens, act)


def phantom_uniform_box(dims=(32, 32, 16), voxel=(4.0, 4.0, 4.0), material=MAT_WATER,
                        density=1.0, source="centre"):
    """Whole grid filled with one material.  source='centre' puts all activity
    in the 8 voxels around the grid centre (a point-like source at the
    centre); 'uniform' fills every voxel."""
    nx, ny, nz = dims
    mat = np.full((nz, ny, nx), material)
    dens = np.full((nz, ny, nx), density)
    act = np.zeros((nz, ny, nx))
    if source == "centre":
        act[nz // 2 - 1:nz // 2 + 1, ny // 2 - 1:ny // 2 + 1, nx // 2 - 1:nx // 2 + 1] = 1.0
    else:
        act[:] = 1.0
    return _finish(dims, voxel, mat, dens, act)


def phantom_torso(dims=(128, 128, 89), voxel=(2.34, 2.34, 2.78), seed=7,
                  semi_axes=(150.0, 100.0), n_spheres=6, sphere_d=(10.0, 37.0),
                  contrast=4.0):
    """Paper-scale synthetic torso: elliptic water cylinder (semi-axes 150 x
    100 mm, full grid length), two lung ellipsoids at 0.3 g/cc, a bone spine
    rod at 1.9 g/cc, and hot spheres whose diameters are evenly spaced over
    ``sphere_d`` at ``contrast``:1 activity, placed on a seeded ring in the
    central slab.  A stand-in with the shapes of the paper's phantoms."""
    rng = np.random.default_rng(seed)
    xx, yy, zz = _centres(dims, voxel)
    a, b = semi_axes
    body = (xx / a) ** 2 + (yy / b) ** 2 <= 1.0
    lung_l = ((xx + 62.0) / 42.0) ** 2 + ((yy - 12.0) / 52.0) ** 2 + (zz / 95.0) ** 2 <= 1.0
    lung_r = ((xx - 62.0) / 42.0) ** 2 + ((yy - 12.0) / 52.0) ** 2 + (zz / 95.0) ** 2 <= 1.0
    lung = body & (lung_l | lung_r)
    spine = body & ((xx / 16.0) ** 2 + ((yy + 68.0) / 16.0) ** 2 <= 1.0)
    mat = np.where(body, MAT_WATER, MAT_VACUUM)
    dens = np.where(body, 1.0, 0.0)
    act = np.where(body, 1.0, 0.0)
    mat = np.where(lung, MAT_LUNG, mat)
    dens = np.where(lung, 0.3, dens)
    act = np.where(lung, 0.3, act)
    mat = np.where(spine, MAT_BONE, mat)
    dens = np.where(spine, 1.9, dens)
    act = np.where(spine, 0.5, act)
    diam = np.linspace(sphere_d[0], sphere_d[1], n_spheres)
    phase = rng.uniform(0, 2 * math.pi)
    for k, d in enumerate(diam):
        ang = phase + 2 * math.pi * k / n_spheres
        cx, cy = 38.0 * math.cos(ang), 30.0 * math.sin(ang) - 10.0
        cz = rng.uniform(-30.0, 30.0)
        sph = (xx - cx) ** 2 + (yy - cy) ** 2 + (zz - cz) ** 2 <= (d / 2.0) ** 2
        sph &= body & ~spine
        mat = np.where(sph, MAT_WATER, mat)
        dens = np.where(sph, 1.0, dens)
        act = np.where(sph, contrast, act)
    return _finish(dims, voxel, mat, dens, act)


def phantom_random_torso(seed, dims, voxel=(3.0, 3.0, 3.0)):
    """Batched-workload torso: seeded ellipse size, random lung/bone inserts
    and lognormal (sigma 0.5) activity contrasts per region."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    xx, yy, zz = _centres(dims, voxel)
    half_x, half_y = 0.5 * nx * voxel[0], 0.5 * ny * voxel[1]
    a = rng.uniform(0.6, 0.92) * half_x
    b = rng.uniform(0.55, 0.9) * min(half_y, a)
    body = (xx / a) ** 2 + (yy / b) ** 2 <= 1.0
    mat = np.where(body, MAT_WATER, MAT_VACUUM)
    dens = np.where(body, 1.0, 0.0)
    act = np.where(body, 1.0, 0.0)
    for _ in range(int(rng.integers(0, 3))):      # lung-like inserts
        cx, cy = rng.uniform(-0.5, 0.5) * a, rng.uniform(-0.3, 0.4) * b
        rx, ry, rz = rng.uniform(0.15, 0.3) * a, rng.uniform(0.2, 0.4) * b, rng.uniform(0.3, 0.5) * nz * voxel[2]
        ins = body & (((xx - cx) / rx) ** 2 + ((yy - cy) / ry) ** 2 + (zz / rz) ** 2 <= 1.0)
        c = rng.lognormal(0.0, 0.5)
        mat, dens, act = np.where(ins, MAT_LUNG, mat), np.where(ins, 0.3, dens), np.where(ins, 0.3 * c, act)
    for _ in range(int(rng.integers(1, 3))):      # bone-like rods
        cx, cy = rng.uniform(-0.3, 0.3) * a, rng.uniform(-0.8, -0.4) * b
        r = rng.uniform(8.0, 18.0)
        ins = body & ((xx - cx) ** 2 + (yy - cy) ** 2 <= r * r)
        mat, dens, act = np.where(ins, MAT_BONE, mat), np.where(ins, 1.9, dens), np.where(ins, 0.5, act)
    for _ in range(int(rng.integers(2, 7))):      # hot/cold spheres
        cx, cy, cz = rng.uniform(-0.5, 0.5) * a, rng.uniform(-0.5, 0.5) * b, rng.uniform(-0.3, 0.3) * nz * voxel[2]
        r = rng.uniform(5.0, 20.0)
        ins = body & ((xx - cx) ** 2 + (yy - cy) ** 2 + (zz - cz) ** 2 <= r * r)
        act = np.where(ins, rng.lognormal(0.0, 0.5) * 2.0, act)
    return _finish(dims, voxel, mat, dens, act)


def batched_phantom_voxel(dims, fov_mm=400.0):
    """Transaxial voxel that keeps an n x n grid's corners inside a 311.8 mm
    detector radius (3 mm up to 133 voxels, then fov_mm / n); 2.78 mm axially."""
    return (min(3.0, fov_mm / dims[0]), min(3.0, fov_mm / dims[1]), 2.78)


def batched_phantom_dims(n=32, seed=11):
    """Uneven phantom sizes from 96x96x64 up to 192x192x120 voxels."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        s = int(rng.integers(96, 193))
        z = int(rng.integers(64, 121))
        out.append((s, s, z))
    return out


def batched_budgets(n=32, seed=13, lo=1e6, hi=1e9):
    """History budgets log-uniform over [lo, hi]."""
    rng = np.random.default_rng(seed)
    return [int(round(10 ** v)) for v in rng.uniform(math.log10(lo), math.log10(hi), n)]


# ---------------------------------------------------------------------------
# Detection-probability LUT
# ---------------------------------------------------------------------------
@dataclass
class Lut:
    n_e: int
    e_min: float           # keV; nodes at bin centres of n_e uniform bins over [e_min, e_max]
    e_max: float
    n_a: int               # transaxial incidence angle bins over [-90, 90] deg
    n_b: int               # axial incidence angle bins over [-90, 90] deg
    n_tpos: int
    n_apos: int
    data: np.ndarray       # f32[n_apos, n_tpos, n_e, n_a, n_b]
    a_min: float = -90.0
    a_max: float = 90.0
    b_min: float = -90.0
    b_max: float = 90.0


def lut_smooth(n_e, n_a, n_b, n_tpos, n_apos, e_min, e_max=511.0, seed=3):
    """Seeded smooth analytic detection probabilities in [0.2, 1]."""
    rng = np.random.default_rng(seed)
    f1, f2, f3 = rng.uniform(0.5, 1.5, 3)
    g = rng.uniform(0, 2 * math.pi, 5)
    e = (np.arange(n_e) + 0.5) / n_e
    a = -1.0 + (np.arange(n_a) + 0.5) * 2.0 / n_a
    b = -1.0 + (np.arange(n_b) + 0.5) * 2.0 / n_b
    t = np.arange(n_tpos) / max(n_tpos, 1)
    z = np.arange(n_apos) / max(n_apos, 1)
    Z, T, E, A, B = np.meshgrid(z, t, e, a, b, indexing="ij")
    h = (np.sin(2 * math.pi * (f1 * E) + g[0]) * np.cos(math.pi * f2 * A + g[1])
         * np.cos(math.pi * f3 * B + g[2])
         * (0.6 + 0.4 * np.cos(2 * math.pi * T + g[3]) * np.cos(2 * math.pi * Z + g[4])))
    p = 0.2 + 0.8 * 0.5 * (1.0 + h)
    return Lut(n_e, float(e_min), float(e_max), n_a, n_b, n_tpos, n_apos,
               np.ascontiguousarray(p, dtype=np.float32))


def lut_histograms(lut, counts=200.0, seed=11):
    """Synthetic stand-ins for the two histograms a LUT is made from (Sec.
    2.2.2): photons reaching the detection cylinder per LUT bin (Poisson,
    mean `counts` times a seeded factor in [0.5, 1.5)) and those of them
    detected (binomial at the LUT's probability)."""
    rng = np.random.default_rng(seed)
    incident = rng.poisson(counts * rng.uniform(0.5, 1.5, lut.data.shape))
    detected = rng.binomial(incident, lut.data.astype(np.float64))
    return incident, detected


def lut_reduced(lut, incident, detected, keep):
    """A lower-dimensional LUT (Sec. 2.2.2): both histograms summed over the
    axes not in `keep` (of "e", "a", "b", "t", "z": energy, transaxial and
    axial angle, transaxial and axial position), then divided; 0 where no
    photon arrived.  A dropped axis keeps one bin."""
    axes = {"z": 0, "t": 1, "e": 2, "a": 3, "b": 4}
    drop = tuple(v for k, v in axes.items() if k not in keep)
    inc = incident.sum(axis=drop, keepdims=True).astype(np.float64)
    det = detected.sum(axis=drop, keepdims=True).astype(np.float64)
    p = np.where(inc > 0, det / np.maximum(inc, 1.0), 0.0)
    n_apos, n_tpos, n_e, n_a, n_b = p.shape
    return Lut(n_e, lut.e_min, lut.e_max, n_a, n_b, n_tpos, n_apos, np.ascontiguousarray(p, dtype=np.float32),
               lut.a_min, lut.a_max, lut.b_min, lut.b_max)


def lut_tiny(scanner):
    return lut_smooth(16, 8, 8, scanner.n_tpos, scanner.n_apos, scanner.e_lo)


def lut_signa(scanner):
    return lut_smooth(64, 32, 32, scanner.n_tpos, scanner.n_apos, scanner.e_lo)


# ---------------------------------------------------------------------------
# Sinogram-shaped inputs
# ---------------------------------------------------------------------------
def sensitivity_uniform(shape, seed=1, lo=0.5, hi=1.5):
    """Uniform-random sensitivity sinogram in [lo, hi) (f64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape)


def sparse_accumulator(n_bins, n_nonzero, seed=5, q_max=1 << 40):
    """Sparse synthetic fixed-point accumulator: sorted unique bin indices and
    int64 values (for finalize tests at full size)."""
    rng = np.random.default_rng(seed)
    idx = np.unique(rng.integers(0, n_bins, size=n_nonzero, dtype=np.int64))
    val = rng.integers(1, q_max, size=idx.size, dtype=np.int64)
    return idx, val
