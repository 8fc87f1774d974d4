"""FP64 oracle of the sinogram post-processing (numpy).

TEST INFRASTRUCTURE (see the package docstring): only tests, the smoke check
and the benchmark's CPU-baseline leg use this module.

* Sensitivity multiply (Sec. 2.2.4): the scatter estimate is the LUT-weighted
  scatter sinogram times the scatter-sensitivity sinogram.
* Smoothing (Sec. 2.3.2): multiply by the smoothing-normalisation sinogram,
  Gaussian-smooth, divide by the same sinogram, then multiply by the
  sensitivity sinogram.  Smoothing is separable along the radial, view and
  axial-within-segment directions (the paper's radial / angular / planar
  FWHMs); each TOF bin is smoothed on its own.

Readings where the paper is silent: kernel truncated at ceil(4 sigma), weights
normalised to sum 1; boundaries reflect about the edge (half-sample
symmetric: -1 -> 0, n -> n-1, repeated periodically for short axes); the view
axis is not wrapped; a plane's axial neighbours are the planes of the same
ring difference rb - ra at ra +- 1 (one ring pitch per planar bin); a zero
normalisation value gives 0.

Sinogram layout [plane][view][radial][tof], plane = ra * n_rings + rb.
Pinned by tests/test_oracle_finalize.py (delta response, mass conservation,
separable == brute-force 3D, elementwise multiply).
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_weights(sigma):
    """Normalised Gaussian taps for offsets -K..K, K = ceil(4 sigma)."""
    if sigma is None or sigma <= 0:
        return np.ones(1)
    K = int(math.ceil(4.0 * sigma))
    k = np.arange(-K, K + 1, dtype=np.float64)
    g = np.exp(-0.5 * (k / sigma) ** 2)
    return g / g.sum()


def reflect_index(m, n):
    """Half-sample symmetric reflection of integer index m into [0, n)."""
    m = np.mod(np.asarray(m), 2 * n)
    return np.where(m >= n, 2 * n - 1 - m, m)


def segment_planes(n_rings):
    """For each ring difference d = rb - ra (from -(n-1) to n-1), the plane
    indices of that segment ordered by ra."""
    segs = []
    for d in range(-(n_rings - 1), n_rings):
        ras = range(max(0, -d), min(n_rings, n_rings - d))
        segs.append(np.array([ra * n_rings + (ra + d) for ra in ras], dtype=np.int64))
    return segs


def _smooth_axis(x, axis, sigma):
    g = gaussian_weights(sigma)
    if g.size == 1:
        return x.copy()
    K = g.size // 2
    n = x.shape[axis]
    idx = np.arange(n)
    out = np.zeros_like(x)
    for j, k in enumerate(range(-K, K + 1)):
        out += g[j] * np.take(x, reflect_index(idx + k, n), axis=axis)
    return out


def smooth(x, n_rings, sigma):
    """Separable Gaussian smoothing of x[plane, view, rad, tof] with
    sigma = (radial, view, axial) in bins: radial, then view, then axial
    within each ring-difference segment."""
    s_rad, s_view, s_ax = sigma
    y = _smooth_axis(x, 2, s_rad)
    y = _smooth_axis(y, 1, s_view)
    out = np.empty_like(y)
    for planes in segment_planes(n_rings):
        out[planes] = _smooth_axis(y[planes], 0, s_ax)
    return out


def _lor_broadcast(a, shape):
    """Per-LOR (plane, view, rad) inputs apply to every TOF bin."""
    if a is None:
        return None
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 3:
        return a[..., None]
    return a.reshape(shape)


def finalize(acc, n_rings, sens=None, norm=None, sigma=None, scale=1.0,
             smooth_before_sensitivity=True):
    """Scatter estimate from the int64 fixed-point accumulator.

    x = acc * (scale * 2^-32); with smoothing:
      x = smooth(x * norm) / norm   (0 where norm == 0)
    and out = x * sens.  With ``smooth_before_sensitivity`` False the
    sensitivity multiply comes first and the smoothing acts on its product.
    sens/norm: None, per-LOR [plane, view, rad] or full [plane, view, rad, tof].
    """
    acc = np.asarray(acc)
    shape = acc.shape
    c = math.ldexp(scale, -32)
    x = acc.astype(np.float64) * c
    S = _lor_broadcast(sens, shape)
    Nn = _lor_broadcast(norm, shape)
    if not smooth_before_sensitivity and S is not None:
        x = x * S
    if sigma is not None:
        if Nn is not None:
            x = x * Nn
        x = smooth(x, n_rings, sigma)
        if Nn is not None:
            safe = np.where(Nn != 0, Nn, 1.0)
            x = np.where(Nn != 0, x / safe, 0.0)
    if smooth_before_sensitivity and S is not None:
        x = x * S
    return x


def finalize_at(bins, shape, n_rings, acc_at, sens_at=None, norm_at=None, sigma=None,
                scale=1.0, smooth_before_sensitivity=True):
    """The same estimate at selected flat bin indices only, written as the
    brute-force 3D product-kernel sum (for full-size sinograms).

    acc_at(flat) -> int64 values; sens_at / norm_at(flat) -> f64 values (their
    per-LOR or per-bin indexing is the caller's).  Mathematically equal to
    ``finalize`` (separable sums factor)."""
    bins = np.asarray(bins, dtype=np.int64)
    n_planes, n_views, n_rad, n_tof = shape
    t = bins % n_tof
    r = (bins // n_tof) % n_rad
    v = (bins // (n_tof * n_rad)) % n_views
    p = bins // (n_tof * n_rad * n_views)
    c = math.ldexp(scale, -32)

    def x_at(flat):
        x = acc_at(flat).astype(np.float64) * c
        if not smooth_before_sensitivity and sens_at is not None:
            x = x * sens_at(flat)
        if sigma is not None and norm_at is not None:
            x = x * norm_at(flat)
        return x

    if sigma is None:
        x = x_at(bins)
    else:
        g1, g2, g3 = (gaussian_weights(s) for s in sigma)
        K1, K2, K3 = g1.size // 2, g2.size // 2, g3.size // 2
        # axial neighbours: plane within its ring-difference segment
        ra, rb = p // n_rings, p % n_rings
        d = rb - ra
        ra_lo = np.maximum(0, -d)
        seg_len = n_rings - np.abs(d)
        j = ra - ra_lo
        k3 = np.arange(-K3, K3 + 1)
        jj = reflect_index(j[:, None] + k3[None, :], seg_len[:, None])
        ra_n = ra_lo[:, None] + jj
        planes = ra_n * n_rings + (ra_n + d[:, None])                      # (S, 2K3+1)
        views = reflect_index(v[:, None] + np.arange(-K2, K2 + 1)[None, :], n_views)   # (S, 2K2+1)
        rads = reflect_index(r[:, None] + np.arange(-K1, K1 + 1)[None, :], n_rad)      # (S, 2K1+1)
        flat = (((planes[:, :, None, None] * n_views + views[:, None, :, None]) * n_rad
                 + rads[:, None, None, :]) * n_tof + t[:, None, None, None])
        xv = x_at(flat.ravel()).reshape(flat.shape)
        w = g3[None, :, None, None] * g2[None, None, :, None] * g1[None, None, None, :]
        x = (xv * w).sum(axis=(1, 2, 3))
        if norm_at is not None:
            nb = norm_at(bins)
            x = np.where(nb != 0, x / np.where(nb != 0, nb, 1.0), 0.0)
    if smooth_before_sensitivity and sens_at is not None:
        x = x * sens_at(bins)
    return x


# ---------------------------------------------------------------------------
# Post-processing beyond the estimate (Sec. 2.2.4, 2.3.2, 4)
# ---------------------------------------------------------------------------
def mash(s, view_factor=1, tof_factor=1):
    """Mashing (Sec. 4 lists it as a way to need fewer counts): adjacent
    views and adjacent TOF bins are summed, [p][v][r][t] ->
    [p][v / view_factor][r][t / tof_factor]."""
    p, v, r, t = s.shape
    if v % view_factor or t % tof_factor:
        raise ValueError("factors must divide the view and TOF counts")
    return s.reshape(p, v // view_factor, view_factor, r, t // tof_factor, tof_factor).sum(axis=(2, 5))


def span_segments(n_rings, span):
    """Segments of span mashing (Sec. 4 names mashing without details; the
    usual Michelogram span is the reading): ring differences d = rb - ra in
    groups of `span` (odd) consecutive values, segment k holding
    [k span - (span-1)/2, k span + (span-1)/2], k = -K..K.  Returns
    [(k, d_lo, d_hi, zs)]: d clipped to the ring range, and zs the axial sums
    z = ra + rb that some plane of the segment has (from the segment's
    smallest |d| to 2 n - 2 minus it; every other one when the segment holds
    a single ring difference)."""
    if span < 1 or span % 2 == 0:
        raise ValueError("span must be odd and >= 1")
    h = (span - 1) // 2
    kmax = (n_rings - 1 + h) // span
    out = []
    for k in range(-kmax, kmax + 1):
        d_lo, d_hi = max(k * span - h, -(n_rings - 1)), min(k * span + h, n_rings - 1)
        m = 0 if d_lo <= 0 <= d_hi else min(abs(d_lo), abs(d_hi))
        step = 1 if d_hi > d_lo else 2
        out.append((k, d_lo, d_hi, list(range(m, 2 * n_rings - 1 - m, step))))
    return out


def span_mash(s, n_rings, span):
    """Span mashing of a sinogram [plane][view][rad][tof] (plane = ra n + rb):
    output plane (k, z) is the sum of every input plane (ra, rb) whose ring
    difference lies in segment k and whose ra + rb = z; segments in order
    k = -K..K, each segment's planes by z ascending.  Brute force over the
    input planes; integer input gives exact sums."""
    index, total = {}, 0
    for k, _, _, zs in span_segments(n_rings, span):
        for z in zs:
            index[(k, z)] = total
            total += 1
    out = np.zeros((total,) + s.shape[1:], dtype=s.dtype)
    h = (span - 1) // 2
    for ra in range(n_rings):
        for rb in range(n_rings):
            d = rb - ra
            k = (abs(d) + h) // span * (1 if d >= 0 else -1)
            out[index[(k, ra + rb)]] += s[ra * n_rings + rb]
    return out


def _view_rad(n, a, b, rad_off):
    """View and kept-radial index of the LOR between crystals a < b (the
    integer LOR formula of the binning)."""
    f = a + b
    s = np.where(f >= n, -1, 1)
    f = np.where(f >= n, f - n, f)
    return f >> 1, s * (n // 2 - (b - a)) + n // 2 - 1 - rad_off


def rotational_average(s, n_crystals, n_rings, step, average=True):
    """Average over the scanner's rotational symmetries (Sec. 2.2.4 exploits
    14 of them for the sensitivity sinograms).  Rotating the ring by a whole
    module of `step` crystals maps it onto itself; the n / step rotations
    form a group whose orbit of an LOR visits n / (2 step) views of a
    180-degree sinogram (14 for 448 crystals in 16-crystal modules), each
    twice: the half turn maps a bin to its radial mirror.  Rotation by c
    crystals maps the LOR (a, b, ring_a, ring_b, delta) to (a + c, b + c)
    mod n; when that reverses the crystal order, the rings swap roles and the
    TOF coordinate changes sign (bin t -> n_tof - 1 - t).  Brute force over
    every crystal pair with the forward LOR formula.  average=False returns
    the sum over the rotations (exact for an int64 fixed-point sinogram)."""
    if n_crystals % step:
        raise ValueError("step must divide n_crystals")
    n_rot = n_crystals // step
    n, nr = n_crystals, n_rings
    p_, v_, r_, t_ = s.shape
    rad_off = (n - 1 - r_) // 2
    a, b = np.triu_indices(n, 1)
    v0, r0 = _view_rad(n, a, b, rad_off)
    keep = (r0 >= 0) & (r0 < r_)
    a, b, v0, r0 = a[keep], b[keep], v0[keep], r0[keep]
    ra, rb = np.divmod(np.arange(p_), nr)
    swapped = rb * nr + ra
    out = np.zeros(s.shape, dtype=np.int64 if (s.dtype.kind == "i" and not average) else np.float64)
    for k in range(n_rot):
        c = k * step
        a2, b2 = (a + c) % n, (b + c) % n
        flip = a2 > b2
        lo, hi = np.minimum(a2, b2), np.maximum(a2, b2)
        v2, r2 = _view_rad(n, lo, hi, rad_off)
        if np.any((r2 < 0) | (r2 >= r_)):
            raise ValueError("a rotation leaves the kept radial range")
        for fl in (False, True):
            m = flip == fl
            src = s[swapped][:, v2[m], r2[m], ::-1] if fl else s[:, v2[m], r2[m], :]
            out[:, v0[m], r0[m], :] += src
    return out / n_rot if average else out


def norm_from_sinogram(s, n_rings, sigma):
    """Smoothing-normalisation sinogram (Sec. 2.3.2): a heavily smoothed
    copy of a sinogram divided by the sinogram itself; 0 where it is 0."""
    sm = smooth(s.astype(np.float64), n_rings, sigma)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(s != 0, sm / np.where(s != 0, s, 1.0), 0.0)
