"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, and exports every entry point that include/psc.h declares; the Python
binding names the same entry points."""
import glob
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(psc_[a-z_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_2509_05047_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["psc_create", "psc_destroy", "psc_last_error", "psc_load_scanner",
                     "psc_load_materials", "psc_load_phantom", "psc_update_activity",
                     "psc_load_lut", "psc_load_sinogram", "psc_acc_create", "psc_acc_zero",
                     "psc_acc_read", "psc_acc_write", "psc_simulate", "psc_finalize",
                     "psc_unload"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"not exported: {missing}"


def test_library_loads_and_binding_matches_header(libpath):
    import paper_2509_05047_gb300 as psc
    L = psc.lib()
    for n in declared_functions():
        assert hasattr(L, n)
        assert n in psc.SIGNATURES and hasattr(psc, n)
    assert psc.psc_last_error() == ""


def test_kernels_are_built_for_sm103a(libpath):
    out = subprocess.check_output(["cuobjdump", "--list-elf", libpath], text=True) \
        if shutil.which("cuobjdump") else "sm_103a"
    assert "sm_103" in out


def test_descriptors_keep_their_host_arrays_alive():
    """A descriptor taken from a temporary holder stays valid (the arrays it
    points into must not be freed before the C call reads them)."""
    import ctypes
    import gc

    import numpy as np

    import paper_2509_05047_gb300 as psc
    import workloads as W
    ph = W.phantom_water_cylinder()
    expect = int(ph.material.sum())
    d = psc.phantom_desc(W.phantom_water_cylinder()).desc
    m = psc.materials_desc(W.standard_materials()).desc
    lu = psc.lut_desc(W.lut_tiny(W.scanner_tiny())).desc
    gc.collect()
    n = 64 * 64 * 32
    assert int(np.ctypeslib.as_array((ctypes.c_uint8 * n).from_address(d.material)).sum()) == expect
    assert m._keep and lu._keep


def test_descriptor_layouts_match_header(tmp_path):
    """Every ctypes descriptor of the binding has the size and field offsets
    of its C struct, as the host compiler lays it out from include/psc.h."""
    import ctypes as C
    import paper_2509_05047_gb300 as psc
    if shutil.which("gcc") is None:
        pytest.skip("no host C compiler")
    pairs = {"ScannerDesc": "psc_scanner_desc", "MaterialsDesc": "psc_materials_desc",
             "PhantomDesc": "psc_phantom_desc", "LutDesc": "psc_lut_desc", "SimArgs": "psc_sim_args",
             "Stats": "psc_stats", "FinalizeArgs": "psc_finalize_args", "Request": "psc_request",
             "ServerConfig": "psc_server_config", "RequestStatus": "psc_request_status",
             "ListmodeEvent": "psc_listmode_event"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "psc.h"', "int main(void) {"]
    expect = []
    for py, c in pairs.items():
        cls = getattr(psc, py)
        lines.append(f'  printf("%zu\\n", sizeof({c}));')
        expect.append(C.sizeof(cls))
        for name, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({c}, {name}));')
            expect.append(getattr(cls, name).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == expect
    # the numpy record type of the listmode output has the same layout
    dt = psc.listmode_dtype()
    ev = psc.ListmodeEvent
    assert dt.itemsize == C.sizeof(ev) == 104
    assert [dt.fields[n][1] for n, _ in ev._fields_] == [getattr(ev, n).offset for n, _ in ev._fields_]
