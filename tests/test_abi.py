"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/nlfdtd.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2005_06997_gb300 import build, nlfdtd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(nlf_[a-z_0-9]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for need in ("nlf_create", "nlf_set_materials", "nlf_set_shapes", "nlf_set_source", "nlf_set_monitors",
                 "nlf_state_bytes", "nlf_bind_state", "nlf_run", "nlf_sync", "nlf_get_field", "nlf_get_spectra",
                 "nlf_get_dft", "nlf_save_state", "nlf_load_state", "nlf_batch_run", "nlf_last_error",
                 "nlf_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert declared_symbols() <= set(nlfdtd.SIGNATURES), declared_symbols() - set(nlfdtd.SIGNATURES)


def test_library_targets_sm103a_only(lib):
    # the build passes exactly one -gencode for compute_103a / sm_103a
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_validation_without_gpu(lib):
    """nlf_create validates on the host and allocates nothing on the device."""
    L = nlfdtd.load()
    g = nlfdtd.nlf_grid()
    g.nx = g.ny = g.nz = 32
    g.dx, g.courant, g.pml_cells, g.eps_background = 1e-9, 0.5, 6, 1.0
    for a in range(3):
        g.boundary[a] = 1
    h = ctypes.c_void_p()
    assert L.nlf_create(ctypes.byref(g), ctypes.byref(h)) == 0
    L.nlf_destroy(h)
    g.courant = 0.6
    assert L.nlf_create(ctypes.byref(g), ctypes.byref(h)) == -2     # CFL
    g.courant = 0.5
    g.boundary[0] = 2
    assert L.nlf_create(ctypes.byref(g), ctypes.byref(h)) == -1     # only PEC and CPML axes exist
