"""FP64 CPU oracle of the PET scatter Monte Carlo path.

TEST INFRASTRUCTURE: this package is the independent reference that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library (``paper_2509_05047_gb300``) and never imports it.

* ``psc_oracle.c`` (plain C99, FP64) -- emission, transport, detection, LUT
  weighting and binning, one history at a time (Sec. 2.2.1-2.2.3);
* ``sinogram.py`` (numpy, FP64) -- sensitivity multiply (Sec. 2.2.4) and the
  normalised Gaussian smoothing (Sec. 2.3.2).

Parity pinned by ``tests/test_oracle_*.py``: see each function's docstring
for what pins it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from .sinogram import (finalize, finalize_at, gaussian_weights, reflect_index,  # noqa: F401
                       segment_planes, smooth, span_mash, span_segments)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psc_oracle.c")
_LIB = os.path.join(_HERE, "libpsc_oracle.so")

CLASSES = ["absorbed", "lost_axial", "energy_window", "step_limit", "same_crystal",
           "out_of_range", "true", "scatter"]
ABSORBED, LOST_AXIAL, ENERGY_WINDOW, STEP_LIMIT, SAME_CRYSTAL, OUT_OF_RANGE, TRUE, SCATTER = range(8)
DETECTED = 15


def build(force=False):
    """Compile the C oracle in place (gcc, FP64, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "psc_oracle.h"))):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm", "-lpthread"]
    subprocess.check_call(cmd, cwd=_HERE)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Scanner(C.Structure):
    _fields_ = [("radius", C.c_double), ("ring_pitch", C.c_double), ("n_crystals", C.c_int32),
                ("n_rings", C.c_int32), ("module_t", C.c_int32), ("module_a", C.c_int32),
                ("e_lo", C.c_double), ("e_hi", C.c_double), ("n_tof", C.c_int32),
                ("n_rad", C.c_int32), ("tof_bin_mm", C.c_double), ("tof_sigma_mm", C.c_double),
                ("e_res", C.c_double), ("gap_mode", C.c_int32), ("gap_t", C.c_double),
                ("gap_a", C.c_double), ("crystal_depth", C.c_double), ("doi", C.c_double),
                ("mu_block", C.c_double)]


class Materials(C.Structure):
    _fields_ = [("n_mat", C.c_int32), ("n_e", C.c_int32), ("compton", C.c_void_p),
                ("rayleigh", C.c_void_p), ("photo", C.c_void_p), ("kappa", C.c_void_p)]


class Phantom(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double),
                ("material", C.c_void_p), ("density", C.c_void_p)]


class Lut(C.Structure):
    _fields_ = [("n_e", C.c_int32), ("n_a", C.c_int32), ("n_b", C.c_int32),
                ("n_tpos", C.c_int32), ("n_apos", C.c_int32),
                ("e_min", C.c_double), ("e_max", C.c_double), ("a_min", C.c_double),
                ("a_max", C.c_double), ("b_min", C.c_double), ("b_max", C.c_double),
                ("data", C.c_void_p)]


_D3 = C.c_double * 3
_I2 = C.c_int32 * 2
_D2 = C.c_double * 2


class Record(C.Structure):
    _fields_ = [("cls", C.c_int32), ("voxel", C.c_int32), ("view", C.c_int32), ("rad", C.c_int32),
                ("plane", C.c_int32), ("tof", C.c_int32), ("key", C.c_int64), ("q", C.c_int64),
                ("w", C.c_double), ("delta", C.c_double), ("emit", _D3), ("dir", _D3),
                ("status", _I2), ("crystal", _I2), ("ring", _I2), ("n_compton", _I2),
                ("n_rayleigh", _I2), ("n_steps", _I2), ("energy", _D2), ("alpha", _D2),
                ("beta", _D2), ("path", _D2), ("prob", _D2), ("hit", _D3 * 2),
                ("exit_pos", _D3 * 2), ("exit_dir", _D3 * 2), ("c_e_before", C.c_double),
                ("c_e_after", C.c_double), ("c_dir_before", _D3), ("c_dir_after", _D3),
                ("e_det", _D2)]


def _record_dtype():
    """numpy view of Record (same layout, checked against ctypes.sizeof)."""
    fields = []
    for name, ct in Record._fields_:
        if ct in (C.c_int32,):
            fields.append((name, np.int32))
        elif ct in (C.c_int64,):
            fields.append((name, np.int64))
        elif ct in (C.c_double,):
            fields.append((name, np.float64))
        elif ct is _D3:
            fields.append((name, np.float64, (3,)))
        elif ct is _I2:
            fields.append((name, np.int32, (2,)))
        elif ct is _D2:
            fields.append((name, np.float64, (2,)))
        else:  # _D3 * 2
            fields.append((name, np.float64, (2, 3)))
    dt = np.dtype(fields, align=True)
    assert dt.itemsize == C.sizeof(Record), (dt.itemsize, C.sizeof(Record))
    return dt


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_alias_build.argtypes = [P, C.c_int64, P, P]
        L.orc_alias_build.restype = C.c_int
        L.orc_majorant.argtypes = [P, P, P]
        L.orc_simulate.argtypes = [P, P, P, P, P, P, C.c_uint64, C.c_uint64, C.c_uint64,
                                   C.c_int32, C.c_int32, P, P, P, P, P, P, P]
        L.orc_simulate.restype = C.c_int
        L.orc_sample_compton.argtypes = [C.c_double, C.c_uint64, C.c_int64, P, P]
        L.orc_sample_rayleigh.argtypes = [C.c_double, C.c_double, C.c_uint64, C.c_int64, P]
        L.orc_lut_prob.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_int32, C.c_int32]
        L.orc_lut_prob.restype = C.c_double
        L.orc_detect.argtypes = [P, P, P, C.c_double, P, P, P, P, P, P]
        L.orc_detect.restype = C.c_int
        L.orc_bin.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                              P, P, P, P, P]
        L.orc_bin.restype = C.c_int
        L.orc_place.argtypes = [P, P, P, P, P, P, P, P, P, P]
        L.orc_place.restype = C.c_int
        L.orc_edge_prob.argtypes = [P, C.c_double, C.c_double, C.c_double]
        L.orc_edge_prob.restype = C.c_double
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ----------------------------------------------------------------------------
# struct marshalling from workloads.* objects
# ----------------------------------------------------------------------------
class _Keep:
    """Holds the numpy buffers a ctypes struct points into."""

    def __init__(self, struct, *arrays):
        self.struct = struct
        self.arrays = arrays

    def ref(self):
        return C.byref(self.struct)


def scanner_struct(sc):
    return _Keep(Scanner(sc.radius, sc.ring_pitch, sc.n_crystals, sc.n_rings, sc.module_t,
                         sc.module_a, sc.e_lo, sc.e_hi, sc.n_tof, sc.n_rad, sc.tof_bin_mm,
                         sc.tof_sigma_mm, getattr(sc, "e_res", 0.0), getattr(sc, "gap_mode", 0),
                         getattr(sc, "gap_t", 0.0), getattr(sc, "gap_a", 0.0),
                         getattr(sc, "crystal_depth", 25.0), getattr(sc, "doi", 7.0),
                         getattr(sc, "mu_block", 0.0869)))


def materials_struct(mats):
    comp = np.ascontiguousarray(np.stack([m.compton for m in mats]), dtype=np.float64)
    rayl = np.ascontiguousarray(np.stack([m.rayleigh for m in mats]), dtype=np.float64)
    phot = np.ascontiguousarray(np.stack([m.photo for m in mats]), dtype=np.float64)
    kap = np.ascontiguousarray([m.kappa for m in mats], dtype=np.float64)
    s = Materials(len(mats), comp.shape[1], _ptr(comp).value, _ptr(rayl).value,
                  _ptr(phot).value, _ptr(kap).value)
    return _Keep(s, comp, rayl, phot, kap)


def phantom_struct(ph):
    mat = np.ascontiguousarray(ph.material, dtype=np.uint8)
    den = np.ascontiguousarray(ph.density, dtype=np.float32)
    nx, ny, nz = ph.dims
    s = Phantom(nx, ny, nz, *ph.voxel, *ph.origin, _ptr(mat).value, _ptr(den).value)
    return _Keep(s, mat, den)


def lut_struct(lut):
    if lut is None:
        return None
    data = np.ascontiguousarray(lut.data, dtype=np.float32)
    s = Lut(lut.n_e, lut.n_a, lut.n_b, lut.n_tpos, lut.n_apos, lut.e_min, lut.e_max,
            lut.a_min, lut.a_max, lut.b_min, lut.b_max, _ptr(data).value)
    return _Keep(s, data)


# ----------------------------------------------------------------------------
# entry points
# ----------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al. 2011).  Pinned by the published
    known-answer vectors in tests/golden/philox4x32_10_kat.txt."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def alias_build(activity):
    """Vose alias table (prob f64, alias i32).  Pinned by the exact
    reconstruction identity and a chi-square of sampled voxel counts."""
    a = np.ascontiguousarray(activity, dtype=np.float32).ravel()
    prob = np.zeros(a.size, dtype=np.float64)
    alias = np.zeros(a.size, dtype=np.int32)
    rc = lib().orc_alias_build(_ptr(a), a.size, _ptr(prob), _ptr(alias))
    if rc != 0:
        raise ValueError("activity must be finite, non-negative, with a positive sum")
    return prob, alias


def majorant(mats, phantom):
    m = materials_struct(mats)
    p = phantom_struct(phantom)
    out = np.zeros(m.arrays[0].shape[1], dtype=np.float64)
    lib().orc_majorant(m.ref(), p.ref(), _ptr(out))
    return out


def simulate(scanner, mats, phantom, lut, seed, first, n, bin_mask=1, threads=1,
             records=False, acc=False, alias=None):
    """Simulate histories [first, first+n).  Returns a dict with per-history
    ``cls`` (int8), ``key`` (int64, -1 unless true/scatter), ``q`` (int64
    fixed-point weight), ``w`` (f64 weight), class ``counts`` and, on
    request, the dense ``acc`` sinogram (int64, scanner.shape) and the full
    listmode ``rec`` (structured numpy array)."""
    if alias is None:
        alias = alias_build(phantom.activity)
    prob, aidx = alias
    s = scanner_struct(scanner)
    m = materials_struct(mats)
    p = phantom_struct(phantom)
    lu = lut_struct(lut)
    cls = np.zeros(n, dtype=np.int8)
    key = np.zeros(n, dtype=np.int64)
    q = np.zeros(n, dtype=np.int64)
    w = np.zeros(n, dtype=np.float64)
    rec = np.zeros(n, dtype=_record_dtype()) if records else None
    a = np.zeros(scanner.n_bins, dtype=np.int64) if acc else None
    counts = np.zeros(8, dtype=np.uint64)
    rc = lib().orc_simulate(s.ref(), m.ref(), p.ref(), _ptr(prob), _ptr(aidx),
                            lu.ref() if lu else None, seed, first, n, bin_mask, threads,
                            _ptr(cls), _ptr(key), _ptr(q), _ptr(w), _ptr(rec), _ptr(a),
                            _ptr(counts))
    if rc != 0:
        raise ValueError("invalid oracle input")
    out = {"cls": cls, "key": key, "q": q, "w": w, "counts": counts.astype(np.int64)}
    if records:
        out["rec"] = rec
    if acc:
        out["acc"] = a.reshape(scanner.shape)
    return out


def sample_compton(e, seed, n):
    """(cos theta, E') of n independent Compton events at energy e (Kahn's
    method).  Pinned by E' = E/(1 + (E/511)(1 - cos)) and a chi-square
    against the closed-form Klein-Nishina distribution."""
    c = np.zeros(n)
    eo = np.zeros(n)
    lib().orc_sample_compton(float(e), seed, n, _ptr(c), _ptr(eo))
    return c, eo


def sample_rayleigh(e, kappa, seed, n):
    """cos theta of n Rayleigh events.  Pinned by the Thomson closed form
    (kappa = 0) and the closed-form form-factor density (kappa > 0)."""
    c = np.zeros(n)
    lib().orc_sample_rayleigh(float(e), float(kappa), seed, n, _ptr(c))
    return c


def lut_prob(lut, e, alpha, beta, tpos, apos):
    """Multilinear LUT probability.  Pinned by node values and exact
    reproduction of multilinear functions."""
    lu = lut_struct(lut)
    return lib().orc_lut_prob(lu.ref() if lu else None, e, alpha, beta, tpos, apos)


def detect(scanner, pos, direction, e=511.0):
    """Detection of one photon.  Returns (status, crystal, ring, hit, alpha,
    beta, dist).  Pinned by hand-built rays with known hits."""
    s = scanner_struct(scanner)
    p = np.ascontiguousarray(pos, dtype=np.float64)
    d = np.ascontiguousarray(direction, dtype=np.float64)
    cr, rg = C.c_int32(), C.c_int32()
    hit = np.zeros(3)
    al, be, di = C.c_double(), C.c_double(), C.c_double()
    st = lib().orc_detect(s.ref(), _ptr(p), _ptr(d), e, C.byref(cr), C.byref(rg), _ptr(hit),
                          C.byref(al), C.byref(be), C.byref(di))
    return st, cr.value, rg.value, hit, al.value, be.value, di.value


def bin_lor(scanner, ca, cb, ra, rb, delta):
    """(status, plane, view, rad, tof, key) of an LOR; ca < cb.  Pinned by
    brute force over all crystal pairs against the continuous geometry."""
    s = scanner_struct(scanner)
    pl, vw, rd, tf = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    k = C.c_int64()
    st = lib().orc_bin(s.ref(), ca, cb, ra, rb, float(delta), C.byref(pl), C.byref(vw),
                       C.byref(rd), C.byref(tf), C.byref(k))
    return st, pl.value, vw.value, rd.value, tf.value, k.value


def place(scanner, hit):
    """(flags, tpos, apos, crystal, ring, xt, xa, bt, ba) of a detector hit
    on a scanner with gaps (flags: 1 transaxial gap, 2 axial gap)."""
    s = scanner_struct(scanner)
    h = np.ascontiguousarray(hit, dtype=np.float64)
    ints = [C.c_int32() for _ in range(6)]
    xt, xa = C.c_double(), C.c_double()
    tp, ap, cr, rg, bt, ba = ints
    fl = lib().orc_place(s.ref(), _ptr(h), C.byref(tp), C.byref(ap), C.byref(cr), C.byref(rg),
                         C.byref(xt), C.byref(xa), C.byref(bt), C.byref(ba))
    return fl, tp.value, ap.value, cr.value, rg.value, xt.value, xa.value, bt.value, ba.value


def edge_prob(scanner, x0, theta_deg, gap):
    """Probability of assignment to the negative-offset block of a gap."""
    s = scanner_struct(scanner)
    return lib().orc_edge_prob(s.ref(), float(x0), float(theta_deg), float(gap))
