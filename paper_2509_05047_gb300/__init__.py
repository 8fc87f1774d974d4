"""Python binding of libpsc, the GB300 PET scatter Monte Carlo library.

Thin ctypes marshalling over the C ABI in ``include/psc.h``: every function
here has the name of the C entry point it calls and does no computation of
its own.  Device buffers are passed as integer device pointers (for example
``tensor.data_ptr()`` of a CUDA torch tensor) and streams as integer
``cudaStream_t`` handles (``torch.cuda.current_stream().cuda_stream``).
Failures raise :class:`PscError` carrying the library's error code and
message.  The library must have been built (``build.build()``); importing the
binding without it fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
# PSC_LIBRARY=debug loads the bounds-checked debug build (libpsc_debug.so)
LIB_PATH = os.path.join(_HERE, "libpsc_debug.so" if os.environ.get("PSC_LIBRARY") == "debug" else "libpsc.so")

PSC_OK, PSC_EINVAL, PSC_ENOMEM, PSC_ENOTFOUND, PSC_ETIMEOUT, PSC_EDEVICE, PSC_EOVERFLOW = (
    0, -1, -2, -3, -4, -5, -6)
PSC_LUT_F32, PSC_LUT_F16, PSC_LUT_BF16 = 0, 1, 2
PSC_BIN_SCATTER, PSC_BIN_TRUES = 1, 2
CLASSES = ["absorbed", "lost_axial", "energy_window", "step_limit", "same_crystal",
           "out_of_range", "true", "scatter"]


class PscError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"psc error {code}: {msg}")
        self.code = code


class ScannerDesc(C.Structure):
    _fields_ = [("radius", C.c_double), ("ring_pitch", C.c_double), ("n_crystals", C.c_int32),
                ("n_rings", C.c_int32), ("module_t", C.c_int32), ("module_a", C.c_int32),
                ("e_lo", C.c_double), ("e_hi", C.c_double), ("n_tof", C.c_int32),
                ("n_rad", C.c_int32), ("tof_bin_mm", C.c_double), ("tof_sigma_mm", C.c_double),
                ("e_res_fwhm", C.c_double), ("gap_mode", C.c_int32), ("gap_t_mm", C.c_double),
                ("gap_a_mm", C.c_double), ("crystal_depth_mm", C.c_double), ("doi_mm", C.c_double),
                ("mu_block", C.c_double)]


class MaterialsDesc(C.Structure):
    _fields_ = [("n_mat", C.c_int32), ("n_e", C.c_int32), ("compton", C.c_void_p),
                ("rayleigh", C.c_void_p), ("photo", C.c_void_p), ("kappa", C.c_void_p)]


class PhantomDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double),
                ("material", C.c_void_p), ("density", C.c_void_p), ("activity", C.c_void_p)]


class LutDesc(C.Structure):
    _fields_ = [("n_e", C.c_int32), ("n_a", C.c_int32), ("n_b", C.c_int32),
                ("n_tpos", C.c_int32), ("n_apos", C.c_int32), ("e_min", C.c_double),
                ("e_max", C.c_double), ("a_min", C.c_double), ("a_max", C.c_double),
                ("b_min", C.c_double), ("b_max", C.c_double), ("dtype", C.c_int32),
                ("data", C.c_void_p)]


class SimArgs(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("first_history", C.c_uint64), ("n_histories", C.c_uint64),
                ("scanner", C.c_int32), ("phantom", C.c_int32), ("lut", C.c_int32),
                ("acc", C.c_int32), ("bin_mask", C.c_int32), ("block", C.c_int32),
                ("grid", C.c_int32), ("cls_out", C.c_void_p), ("key_out", C.c_void_p),
                ("q_out", C.c_void_p), ("lm_out", C.c_void_p), ("lm_count", C.c_void_p),
                ("lm_capacity", C.c_uint64)]


class ListmodeEvent(C.Structure):
    """One coincidence of the listmode debug output (psc_listmode_event)."""
    _fields_ = [("history", C.c_uint64), ("q", C.c_int64), ("voxel", C.c_int32), ("cls", C.c_int32),
                ("delta_mm", C.c_float), ("energy_kev", C.c_float * 2), ("phi", C.c_float * 2),
                ("z_mm", C.c_float * 2), ("dir", (C.c_float * 3) * 2), ("crystal", C.c_int32 * 2),
                ("ring", C.c_int32 * 2), ("n_scatter", C.c_uint16 * 2), ("rayleigh", C.c_uint8 * 2),
                ("pad", C.c_uint8 * 6)]


def listmode_dtype():
    """numpy dtype with the layout of psc_listmode_event."""
    import numpy as np
    return np.dtype([("history", "<u8"), ("q", "<i8"), ("voxel", "<i4"), ("cls", "<i4"),
                     ("delta_mm", "<f4"), ("energy_kev", "<f4", (2,)), ("phi", "<f4", (2,)),
                     ("z_mm", "<f4", (2,)), ("dir", "<f4", (2, 3)), ("crystal", "<i4", (2,)),
                     ("ring", "<i4", (2,)), ("n_scatter", "<u2", (2,)), ("rayleigh", "u1", (2,)),
                     ("pad", "u1", (6,))])


class Stats(C.Structure):
    _fields_ = [("class_counts", C.c_uint64 * 8), ("steps", C.c_uint64), ("compton", C.c_uint64),
                ("rayleigh", C.c_uint64), ("photo", C.c_uint64), ("binned", C.c_uint64),
                ("weight_sum", C.c_uint64), ("rng_blocks", C.c_uint64), ("tries", C.c_uint64),
                ("detected", C.c_uint64), ("atomics", C.c_uint64), ("grid", C.c_int32),
                ("block", C.c_int32)]

    def as_dict(self):
        d = {k: int(v) for k, v in zip(CLASSES, self.class_counts)}
        for f in ("steps", "compton", "rayleigh", "photo", "binned", "weight_sum", "rng_blocks",
                  "tries", "detected", "atomics", "grid", "block"):
            d[f] = int(getattr(self, f))
        return d


class FinalizeArgs(C.Structure):
    _fields_ = [("acc", C.c_int32), ("sens", C.c_int32), ("norm", C.c_int32),
                ("smooth", C.c_int32), ("sigma", C.c_double * 3), ("scale", C.c_double),
                ("sens_first", C.c_int32), ("seg_lo", C.c_int32), ("seg_hi", C.c_int32)]


class Schedule(C.Structure):
    _fields_ = [("block", C.c_int32), ("grid", C.c_int32), ("chunks_per_cta", C.c_int32),
                ("max_chunk", C.c_int32), ("rate", C.c_double), ("probed", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(C.Structure):
    _fields_ = [("scanner", C.c_int32), ("phantom", C.c_int32), ("lut", C.c_int32),
                ("seed", C.c_uint64), ("first_history", C.c_uint64), ("n_histories", C.c_uint64),
                ("sens", C.c_int32), ("norm", C.c_int32), ("smooth", C.c_int32),
                ("sigma", C.c_double * 3), ("scale", C.c_double), ("sens_first", C.c_int32),
                ("out", C.c_void_p), ("activity", C.c_void_p)]


class ServerConfig(C.Structure):
    _fields_ = [("max_active", C.c_int32), ("epoch_histories", C.c_uint64),
                ("min_slice", C.c_uint64)]


class RequestStatus(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double)]


PSC_REQ_WAITING, PSC_REQ_ACTIVE, PSC_REQ_FINALIZING, PSC_REQ_DONE, PSC_REQ_FAILED = range(5)

# exported entry points: name -> (restype, argtypes)
_P, _I32, _U64 = C.c_void_p, C.c_int32, C.c_uint64
SIGNATURES = {
    "psc_create": (C.c_int, [C.POINTER(C.c_void_p), _I32, _U64]),
    "psc_destroy": (None, [_P]),
    "psc_check_philox": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "psc_check_curand_philox": (C.c_int, [_U64, _U64, _I32, C.c_void_p]),
    "psc_peak_random_atomics": (C.c_int, [C.c_void_p, _U64, _I32, _I32, _I32, _U64, C.c_void_p]),
    "psc_peak_random_gather": (C.c_int, [C.c_void_p, C.c_uint32, _I32, _I32, _I32, _U64, C.c_void_p,
                                         C.c_void_p]),
    "psc_host_alloc": (C.c_int, [_U64, C.POINTER(C.c_void_p)]),
    "psc_host_free": (C.c_int, [C.c_void_p]),
    "psc_last_error": (C.c_char_p, []),
    "psc_load_scanner": (C.c_int, [_P, C.POINTER(ScannerDesc), C.POINTER(_I32)]),
    "psc_load_materials": (C.c_int, [_P, C.POINTER(MaterialsDesc), C.POINTER(_I32)]),
    "psc_load_phantom": (C.c_int, [_P, C.POINTER(PhantomDesc), _I32, C.POINTER(_I32)]),
    "psc_update_activity": (C.c_int, [_P, _I32, _P]),
    "psc_phantom_alias": (C.c_int, [_P, _I32, _P, _P]),
    "psc_load_lut": (C.c_int, [_P, C.POINTER(LutDesc), C.POINTER(_I32)]),
    "psc_load_sinogram": (C.c_int, [_P, _I32, _P, _I32, C.POINTER(_I32)]),
    "psc_acc_create": (C.c_int, [_P, _I32, C.POINTER(_I32)]),
    "psc_acc_wrap": (C.c_int, [_P, _I32, _P, C.POINTER(_I32)]),
    "psc_acc_zero": (C.c_int, [_P, _I32, _P]),
    "psc_acc_read": (C.c_int, [_P, _I32, _P, _P]),
    "psc_acc_write": (C.c_int, [_P, _I32, _P, _P]),
    "psc_simulate": (C.c_int, [_P, C.POINTER(SimArgs), C.POINTER(Stats), _P]),
    "psc_simulate_batch": (C.c_int, [_P, C.POINTER(SimArgs), _I32, C.POINTER(Stats), _P]),
    "psc_finalize": (C.c_int, [_P, C.POINTER(FinalizeArgs), _P, _P]),
    "psc_acc_span": (C.c_int, [_P, _I32, _I32, _P, C.POINTER(C.c_int64), _P]),
    "psc_simulate_batch_tuned": (C.c_int, [_P, C.POINTER(SimArgs), _I32, C.POINTER(Schedule), _P]),
    "psc_finalize_host": (C.c_int, [_P, C.POINTER(FinalizeArgs), _P, _P, _P, _P]),
    "psc_finalize_static": (C.c_int, [_P, _I32, _I32, _I32, _I32, _P, _I32, _P, _I32, _P,
                                      C.c_double, _I32, _P, _P]),
    "psc_norm_sinogram": (C.c_int, [_P, _I32, _P, _P, _P]),
    "psc_acc_mash": (C.c_int, [_P, _I32, _I32, _I32, _P, _P]),
    "psc_acc_rotate_sum": (C.c_int, [_P, _I32, _I32, _I32, _P]),
    "psc_unload": (C.c_int, [_P, _I32]),
    "psc_resident_bytes": (_U64, [_P]),
    "psc_phantom_voxels": (C.c_int64, [_P, _I32]),
    "psc_server_start": (C.c_int, [_P, C.POINTER(ServerConfig)]),
    "psc_server_stop": (C.c_int, [_P]),
    "psc_submit": (C.c_int, [_P, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "psc_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(RequestStatus)]),
    "psc_wait": (C.c_int, [_P, C.c_uint64, C.c_int64]),
}

_lib = None


def lib():
    """The loaded libpsc.so, or libpsc_debug.so with PSC_LIBRARY=debug (raises
    if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(paper_2509_05047_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != PSC_OK:
        raise PscError(rc, psc_last_error())
    return rc


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())  # torch tensor


def _stream(s):
    return None if s is None else int(s)


# ---------------------------------------------------------------------------
# C entry points
# ---------------------------------------------------------------------------
def psc_last_error():
    return lib().psc_last_error().decode()


def psc_create(device=0, mem_budget_bytes=0):
    h = C.c_void_p()
    _check(lib().psc_create(C.byref(h), device, mem_budget_bytes))
    return h.value


def psc_destroy(ctx):
    lib().psc_destroy(ctx)


def psc_resident_bytes(ctx):
    return int(lib().psc_resident_bytes(ctx))


def psc_check_philox(ctr_key):
    """The transport kernel's Philox4x32-10 on rows (c0, c1, c2, c3, k0, k1)."""
    a = np.ascontiguousarray(ctr_key, dtype=np.uint32).reshape(-1, 6)
    out = np.zeros((a.shape[0], 4), dtype=np.uint32)
    _check(lib().psc_check_philox(a.ctypes.data, a.shape[0], out.ctypes.data))
    return out


def psc_check_curand_philox(seed, subsequence, n_blocks):
    """cuRAND's Philox4_32_10: n_blocks curand4 draws after curand_init(seed, subsequence, 0)."""
    out = np.zeros((n_blocks, 4), dtype=np.uint32)
    _check(lib().psc_check_curand_philox(seed, subsequence, n_blocks, out.ctypes.data))
    return out


def psc_peak_random_atomics(buf, grid, block, per_thread, seed=1, stream=None):
    """Measurement kernel: random int64 atomic adds into the device tensor buf."""
    _check(lib().psc_peak_random_atomics(_ptr(buf), buf.numel(), grid, block, per_thread, seed,
                                         _stream(stream)))


def psc_peak_random_gather(table, sink, grid, block, per_thread, seed=1, stream=None):
    """Measurement kernel: random 4-byte gathers from the device float tensor table."""
    _check(lib().psc_peak_random_gather(_ptr(table), table.numel(), grid, block, per_thread, seed,
                                        _ptr(sink), _stream(stream)))


def psc_host_alloc(nbytes):
    p = C.c_void_p()
    _check(lib().psc_host_alloc(int(nbytes), C.byref(p)))
    return int(p.value)


def psc_host_free(ptr):
    _check(lib().psc_host_free(C.c_void_p(ptr)))


def host_tensor(shape, dtype=None):
    """A CPU tensor over a psc_host_alloc buffer (page-locked, huge pages),
    freed when the last view of it is collected."""
    import weakref
    import numpy as np
    import torch
    dtype = dtype or torch.float64
    n = 1
    for d in shape:
        n *= int(d)
    nbytes = max(1, n * torch.empty((), dtype=dtype).element_size())
    ptr = psc_host_alloc(nbytes)
    raw = np.ctypeslib.as_array((C.c_uint8 * nbytes).from_address(ptr))
    # at interpreter exit CUDA may be gone before the buffer: the return code is dropped
    weakref.finalize(raw, lambda p=ptr: lib().psc_host_free(C.c_void_p(p)))
    return torch.from_numpy(raw).view(dtype)[:n].view(tuple(shape))


def psc_load_scanner(ctx, desc: ScannerDesc):
    i = C.c_int32()
    _check(lib().psc_load_scanner(ctx, C.byref(desc), C.byref(i)))
    return i.value


def psc_load_materials(ctx, desc: MaterialsDesc):
    i = C.c_int32()
    _check(lib().psc_load_materials(ctx, C.byref(desc), C.byref(i)))
    return i.value


def psc_load_phantom(ctx, desc: PhantomDesc, materials):
    i = C.c_int32()
    _check(lib().psc_load_phantom(ctx, C.byref(desc), materials, C.byref(i)))
    return i.value


def psc_update_activity(ctx, phantom, activity):
    a = np.ascontiguousarray(activity, dtype=np.float32)
    _check(lib().psc_update_activity(ctx, phantom, a.ctypes.data))


def psc_phantom_alias(ctx, phantom, n_vox):
    thr = np.zeros(n_vox, dtype=np.uint32)
    alias = np.zeros(n_vox, dtype=np.int32)
    _check(lib().psc_phantom_alias(ctx, phantom, thr.ctypes.data, alias.ctypes.data))
    return thr, alias


def psc_load_lut(ctx, desc: LutDesc):
    i = C.c_int32()
    _check(lib().psc_load_lut(ctx, C.byref(desc), C.byref(i)))
    return i.value


def psc_load_sinogram(ctx, scanner, host, per_lor):
    h = np.ascontiguousarray(host, dtype=np.float64)
    i = C.c_int32()
    _check(lib().psc_load_sinogram(ctx, scanner, h.ctypes.data, 1 if per_lor else 0, C.byref(i)))
    return i.value


def psc_acc_create(ctx, scanner):
    i = C.c_int32()
    _check(lib().psc_acc_create(ctx, scanner, C.byref(i)))
    return i.value


def psc_acc_wrap(ctx, scanner, device_tensor):
    """An accumulator over a caller-owned int64 device tensor (kept alive by
    the caller until psc_unload)."""
    i = C.c_int32()
    _check(lib().psc_acc_wrap(ctx, scanner, _ptr(device_tensor), C.byref(i)))
    return i.value


def psc_acc_zero(ctx, acc, stream=None):
    _check(lib().psc_acc_zero(ctx, acc, _stream(stream)))


def psc_acc_read(ctx, acc, out, stream=None):
    _check(lib().psc_acc_read(ctx, acc, _ptr(out), _stream(stream)))


def psc_acc_write(ctx, acc, src, stream=None):
    _check(lib().psc_acc_write(ctx, acc, _ptr(src), _stream(stream)))


def psc_simulate(ctx, args: SimArgs, stats=False, stream=None):
    st = Stats() if stats else None
    _check(lib().psc_simulate(ctx, C.byref(args), C.byref(st) if st is not None else None,
                              _stream(stream)))
    return st.as_dict() if st is not None else None


def psc_simulate_batch(ctx, args_list, stats=False, stream=None):
    arr = (SimArgs * len(args_list))(*args_list)
    st = Stats() if stats else None
    _check(lib().psc_simulate_batch(ctx, arr, len(args_list),
                                    C.byref(st) if st is not None else None, _stream(stream)))
    return st.as_dict() if st is not None else None


def psc_simulate_batch_tuned(ctx, args_list, stream=None):
    """psc_simulate_batch with an autotuned launch schedule; returns the
    schedule (dict: block, grid, chunks_per_cta, max_chunk, rate, probed)."""
    arr = (SimArgs * len(args_list))(*args_list)
    sch = Schedule()
    _check(lib().psc_simulate_batch_tuned(ctx, arr, len(args_list), C.byref(sch), _stream(stream)))
    return sch.as_dict()


def psc_finalize(ctx, args: FinalizeArgs, out, stream=None):
    _check(lib().psc_finalize(ctx, C.byref(args), _ptr(out), _stream(stream)))


def psc_finalize_host(ctx, args: FinalizeArgs, work, out_host, stream=None, copy_stream=None):
    """psc_finalize into the device buffer ``work``, each finished part copied
    to ``out_host`` (a host tensor, best from host_tensor) on
    ``copy_stream`` (default: ``stream``)."""
    _check(lib().psc_finalize_host(ctx, C.byref(args), _ptr(work), _ptr(out_host), _stream(stream),
                                   _stream(copy_stream if copy_stream is not None else stream)))


def psc_finalize_static(acc, n_rings, n_crystals, n_rad, n_tof, out, sens=None, sens_per_lor=True,
                        norm=None, norm_per_lor=True, sigma=None, scale=1.0, sens_first=False,
                        stream=None):
    """Allocation-free finalize on caller-owned device arrays (see psc.h)."""
    sig = (C.c_double * 3)(*sigma) if sigma is not None else None
    _check(lib().psc_finalize_static(_ptr(acc), n_rings, n_crystals, n_rad, n_tof, _ptr(sens),
                                     1 if sens_per_lor else 0, _ptr(norm), 1 if norm_per_lor else 0,
                                     sig, scale, 1 if sens_first else 0, _ptr(out), _stream(stream)))


def psc_norm_sinogram(ctx, acc, sigma, out, stream=None):
    """Smoothing-normalisation sinogram smooth(acc) / acc into ``out``."""
    sig = (C.c_double * 3)(*sigma)
    _check(lib().psc_norm_sinogram(ctx, acc, sig, _ptr(out), _stream(stream)))


def psc_acc_span(ctx, acc, span, out=None, stream=None):
    """Span-mash an accumulator into ``out`` (int64 device tensor of
    [planes][views][rad][tof]); returns the number of output planes (out=None
    only queries it)."""
    n = C.c_int64()
    _check(lib().psc_acc_span(ctx, acc, span, _ptr(out), C.byref(n), _stream(stream)))
    return n.value


def psc_acc_mash(ctx, acc, view_factor, tof_factor, out, stream=None):
    """Sum adjacent views / TOF bins of an accumulator into ``out`` (int64)."""
    _check(lib().psc_acc_mash(ctx, acc, view_factor, tof_factor, _ptr(out), _stream(stream)))


def psc_acc_rotate_sum(ctx, acc, step, out_acc, stream=None):
    """Sum of an accumulator over the scanner's module rotations into ``out_acc``."""
    _check(lib().psc_acc_rotate_sum(ctx, acc, step, out_acc, _stream(stream)))


def psc_unload(ctx, obj):
    _check(lib().psc_unload(ctx, obj))


def psc_phantom_voxels(ctx, phantom):
    n = lib().psc_phantom_voxels(ctx, phantom)
    if n < 0:
        _check(int(n))
    return int(n)


def psc_server_start(ctx, max_active=4, epoch_histories=200_000_000, min_slice=0):
    _check(lib().psc_server_start(ctx, C.byref(ServerConfig(max_active, epoch_histories, min_slice))))


def psc_server_stop(ctx):
    _check(lib().psc_server_stop(ctx))


def psc_submit(ctx, req: Request):
    t = C.c_uint64()
    _check(lib().psc_submit(ctx, C.byref(req), C.byref(t)))
    return t.value


def psc_poll(ctx, ticket):
    st = RequestStatus()
    _check(lib().psc_poll(ctx, ticket, C.byref(st)))
    return {"state": st.state, "error": st.error, "t_submit": st.t_submit,
            "t_start": st.t_start, "t_done": st.t_done}


def psc_wait(ctx, ticket, timeout_us=-1):
    """Wait for a request; timeout_us < 0 waits without bound (in 1 s slices
    of the bounded library wait)."""
    if timeout_us >= 0:
        _check(lib().psc_wait(ctx, ticket, timeout_us))
        return
    while True:
        rc = lib().psc_wait(ctx, ticket, 1_000_000)
        if rc != PSC_ETIMEOUT:
            _check(rc)
            return


def request(scanner, phantom, out, n_histories, seed, lut=0, first=0, sens=0, norm=0, sigma=None,
            scale=1.0, sens_first=False, activity=None):
    act = None if activity is None else np.ascontiguousarray(activity, dtype=np.float32)
    s = (C.c_double * 3)(*(sigma if sigma is not None else (0.0, 0.0, 0.0)))
    r = Request(scanner, phantom, lut, seed, first, n_histories, sens, norm,
                1 if sigma is not None else 0, s, scale, 1 if sens_first else 0, _ptr(out),
                None if act is None else act.ctypes.data)
    r._keep = (act,)
    return r


# ---------------------------------------------------------------------------
# marshalling of the ``workloads`` input objects into descriptors
# ---------------------------------------------------------------------------
class _Held:
    """A ctypes descriptor plus the host arrays it points into.  The
    descriptor itself also references the arrays, so ``held.desc`` stays
    valid after the holder is gone."""

    def __init__(self, desc, *arrays):
        desc._keep = arrays
        self.desc = desc
        self.arrays = arrays


def scanner_desc(sc):
    return ScannerDesc(sc.radius, sc.ring_pitch, sc.n_crystals, sc.n_rings, sc.module_t,
                       sc.module_a, sc.e_lo, sc.e_hi, sc.n_tof, sc.n_rad, sc.tof_bin_mm,
                       sc.tof_sigma_mm, getattr(sc, "e_res", 0.0), getattr(sc, "gap_mode", 0),
                       getattr(sc, "gap_t", 0.0), getattr(sc, "gap_a", 0.0),
                       getattr(sc, "crystal_depth", 25.0), getattr(sc, "doi", 7.0),
                       getattr(sc, "mu_block", 0.0869))


def materials_desc(mats):
    comp = np.ascontiguousarray(np.stack([m.compton for m in mats]), dtype=np.float64)
    rayl = np.ascontiguousarray(np.stack([m.rayleigh for m in mats]), dtype=np.float64)
    phot = np.ascontiguousarray(np.stack([m.photo for m in mats]), dtype=np.float64)
    kap = np.ascontiguousarray([m.kappa for m in mats], dtype=np.float64)
    d = MaterialsDesc(len(mats), comp.shape[1], comp.ctypes.data, rayl.ctypes.data,
                      phot.ctypes.data, kap.ctypes.data)
    return _Held(d, comp, rayl, phot, kap)


def phantom_desc(ph):
    mat = np.ascontiguousarray(ph.material, dtype=np.uint8)
    den = np.ascontiguousarray(ph.density, dtype=np.float32)
    act = np.ascontiguousarray(ph.activity, dtype=np.float32)
    nx, ny, nz = ph.dims
    d = PhantomDesc(nx, ny, nz, *ph.voxel, *ph.origin, mat.ctypes.data, den.ctypes.data,
                    act.ctypes.data)
    return _Held(d, mat, den, act)


def lut_desc(lut, dtype=PSC_LUT_F32, ones=False):
    data = None if ones else np.ascontiguousarray(lut.data, dtype=np.float32)
    d = LutDesc(lut.n_e, lut.n_a, lut.n_b, lut.n_tpos, lut.n_apos, lut.e_min, lut.e_max,
                lut.a_min, lut.a_max, lut.b_min, lut.b_max, dtype,
                None if data is None else data.ctypes.data)
    return _Held(d, data)


def sim_args(seed, first, n, scanner, phantom, acc, lut=0, bin_mask=PSC_BIN_SCATTER, block=0,
             grid=0, cls_out=None, key_out=None, q_out=None, lm_out=None, lm_count=None, lm_capacity=0):
    """lm_out: a device uint8 tensor of lm_capacity * 104 bytes for listmode
    records; lm_count: a device int64 tensor of one element (the counter)."""
    return SimArgs(seed, first, n, scanner, phantom, lut, acc, bin_mask, block, grid,
                   _ptr(cls_out), _ptr(key_out), _ptr(q_out), _ptr(lm_out), _ptr(lm_count),
                   int(lm_capacity))


def finalize_args(acc, sens=0, norm=0, sigma=None, scale=1.0, sens_first=False, segments=None):
    """psc_finalize_args; ``segments`` = (lo, hi) finalizes only the planes of
    ring-difference segments [lo, hi) (default: every plane)."""
    s = (C.c_double * 3)(*(sigma if sigma is not None else (0.0, 0.0, 0.0)))
    lo, hi = segments if segments is not None else (0, 0)
    return FinalizeArgs(acc, sens, norm, 1 if sigma is not None else 0, s, scale,
                        1 if sens_first else 0, lo, hi)
