"""Failure detection on the host, without a GPU: the C ABI validates a
problem and plans its state on the host, so malformed or unstable problems
are refused with an NLF_E_* code (and a message) before any device work.

Contexts are built here directly through the binding's structures (the
Solver class insists on a GPU); nlf_bind_state is given a 256-byte aligned
address that is never dereferenced: binding only plans and records it."""
import ctypes as C
import copy

import pytest

from paper_2005_06997_gb300 import build, nlfdtd
from paper_2005_06997_gb300 import workloads as W

E_ARG, E_CFL, E_GEOMETRY, E_OOM, E_STATE = -1, -2, -3, -4, -8
FAKE_PTR = 1 << 40          # aligned, never touched


@pytest.fixture(scope="module")
def L():
    build.build()
    return nlfdtd.load()


def make_ctx(L, prob, with_source=True, with_monitors=True):
    h = C.c_void_p()
    g = nlfdtd.make_grid(prob)
    rc = L.nlf_create(C.byref(g), C.byref(h))
    assert rc == 0
    mats, nm = nlfdtd.make_materials(prob)
    rcs = {"materials": L.nlf_set_materials(h, mats, nm)}
    shp, ns = nlfdtd.make_shapes(prob)
    rcs["shapes"] = L.nlf_set_shapes(h, shp, ns)
    keep = []
    if with_source and prob.get("source") is not None:
        src = nlfdtd.make_source(prob["source"])
        rcs["source"] = L.nlf_set_source(h, C.byref(src))
    if with_monitors and prob.get("monitors") is not None:
        mon, om = nlfdtd.make_monitors(prob["monitors"])
        keep.append(om)
        rcs["monitors"] = L.nlf_set_monitors(h, C.byref(mon))
    return h, rcs


def bind(L, h, nbytes):
    return L.nlf_bind_state(h, C.c_void_p(FAKE_PTR), nbytes)


def base_problem():
    return W.small_sphere(n=36, steps=0, nf=8, K=4)


def test_well_formed_problem_plans(L):
    h, rcs = make_ctx(L, base_problem())
    assert all(v == 0 for v in rcs.values()), rcs
    nb = L.nlf_state_bytes(h)
    assert nb > 0
    assert bind(L, h, nb) == 0
    L.nlf_destroy(h)


def test_bound_buffer_too_small_is_oom(L):
    h, _ = make_ctx(L, base_problem())
    nb = L.nlf_state_bytes(h)
    assert bind(L, h, nb - 1) == E_OOM
    assert b"bound buffer" in L.nlf_last_error(h)
    assert bind(L, h, nb) == 0                   # the refused bind left nothing behind
    L.nlf_destroy(h)


def test_unaligned_bind_is_refused(L):
    h, _ = make_ctx(L, base_problem())
    assert L.nlf_bind_state(h, C.c_void_p(FAKE_PTR + 64), 1 << 30) == E_ARG
    L.nlf_destroy(h)


def test_metal_near_the_tf_surface_is_a_geometry_error(L):
    """Nonlocal metal only inside the total-field region (Sec. III): a sphere
    moved to touch the TF surface is refused, with no device work."""
    prob = base_problem()
    tf_lo = prob["source"]["tf_lo"][0]
    sh = prob["shapes"][0]
    # centre so that the sphere's lowest x cell sits one cell inside the TF box
    sh["c"] = (2 * (tf_lo + 1) + sh["radius"], sh["c"][1], sh["c"][2])
    h, rcs = make_ctx(L, prob, with_monitors=False)
    assert rcs["shapes"] == 0
    assert L.nlf_state_bytes(h) == 0
    assert bind(L, h, 1 << 30) == E_GEOMETRY
    assert b"TF surface" in L.nlf_last_error(h)
    L.nlf_destroy(h)


def test_metal_in_the_cpml_with_a_source_is_a_geometry_error(L):
    prob = base_problem()
    sh = prob["shapes"][0]
    sh["c"] = (2 * 3 + sh["radius"], sh["c"][1], sh["c"][2])      # reaches cell 3, inside the 6-cell CPML
    h, _ = make_ctx(L, prob, with_monitors=False)
    assert bind(L, h, 1 << 30) == E_GEOMETRY
    L.nlf_destroy(h)


def test_absorption_box_must_enclose_the_metal(L):
    prob = base_problem()
    mo = prob["monitors"]
    mo["abs_hi"] = tuple(x - 3 for x in mo["abs_hi"])
    h, rcs = make_ctx(L, prob)
    assert bind(L, h, 1 << 30) == E_GEOMETRY
    assert b"absorption box" in L.nlf_last_error(h)
    L.nlf_destroy(h)


def test_unstable_hydrodynamic_term_is_refused(L):
    """beta dt sqrt(3) / dx > 1 grows without bound (the discrete plasmon
    relation's stability limit): refused at nlf_set_materials."""
    prob = base_problem()
    dt = prob["courant"] * prob["dx"] / W.C0
    beta_lim = prob["dx"] / (dt * 3 ** 0.5)
    ok = copy.deepcopy(prob)
    ok["materials"][0]["beta"] = 0.99 * beta_lim
    ok["materials"][0]["diff"] = 0.0
    h, rcs = make_ctx(L, ok)
    assert rcs["materials"] == 0
    L.nlf_destroy(h)
    bad = copy.deepcopy(prob)
    bad["materials"][0]["beta"] = 1.01 * beta_lim
    bad["materials"][0]["diff"] = 0.0
    h, rcs = make_ctx(L, bad)
    assert rcs["materials"] == E_CFL
    L.nlf_destroy(h)


def test_material_map_ids_beyond_the_table_are_refused(L):
    import numpy as np
    prob = base_problem()
    h, _ = make_ctx(L, prob, with_source=False, with_monitors=False)
    nx, ny, nz = prob["shape"]
    ids = np.zeros((3, nz, ny, nx), dtype=np.uint8)
    ids[0, nz // 2, ny // 2, nx // 2] = 7                  # only one material in the table
    assert L.nlf_set_material_map(h, ids.ctypes.data, 0) == 0
    assert bind(L, h, 1 << 30) == E_ARG
    assert b"exceeds" in L.nlf_last_error(h)
    L.nlf_destroy(h)


def test_monitors_need_a_source_and_sane_sizes(L):
    prob = base_problem()
    h, rcs = make_ctx(L, prob, with_source=False, with_monitors=True)
    assert rcs["monitors"] == E_STATE
    L.nlf_destroy(h)
    h, _ = make_ctx(L, prob, with_monitors=False)
    mon, om = nlfdtd.make_monitors(prob["monitors"])
    mon.decimate_k = 0
    assert L.nlf_set_monitors(h, C.byref(mon)) == E_ARG
    L.nlf_destroy(h)


def test_plane_monitor_outside_the_grid_is_refused(L):
    import numpy as np
    prob = base_problem()
    h, _ = make_ctx(L, prob)
    om = np.array([1e15])
    pm = nlfdtd.nlf_plane_monitor(2, prob["shape"][2], 1, om.ctypes.data_as(C.POINTER(C.c_double)), 4)
    assert L.nlf_set_plane_monitor(h, C.byref(pm)) == E_ARG
    pm = nlfdtd.nlf_plane_monitor(2, 3, 1, om.ctypes.data_as(C.POINTER(C.c_double)), 4)
    assert L.nlf_set_plane_monitor(h, C.byref(pm)) == 0
    L.nlf_destroy(h)


def _grid(n3, pml=6, bc=("cpml",) * 3, courant=0.5):
    g = nlfdtd.nlf_grid()
    g.nx, g.ny, g.nz = n3
    g.dx, g.courant, g.pml_cells, g.eps_background = 1e-9, courant, pml, 1.0
    for a in range(3):
        g.boundary[a] = 1 if bc[a] == "cpml" else 0
    return g


def _create(L, g):
    h = C.c_void_p()
    rc = L.nlf_create(C.byref(g), C.byref(h))
    if rc == 0:
        L.nlf_destroy(h)
    return rc


def test_grid_limits(L):
    """Edge cases of the grid: the smallest grid (8 cells on every axis), the
    thinnest axis a CPML of L cells allows (2 L + 4 cells), the largest grid
    whose 32-bit offsets of three components fit (3 px ny nz < 2^32, px = nx
    rounded up to 8), and one cell past each limit."""
    assert _create(L, _grid((8, 8, 8), bc=("pec",) * 3)) == 0
    assert _create(L, _grid((7, 8, 8), bc=("pec",) * 3)) == E_ARG
    assert _create(L, _grid((16, 16, 16), pml=6)) == 0
    assert _create(L, _grid((15, 16, 16), pml=6)) == E_ARG
    assert _create(L, _grid((16, 16, 16), pml=0)) == E_ARG            # a CPML needs at least one cell
    # 3 px ny nz < 2^32: with px = ny = 1024, nz = 1365 fits, 1366 does not
    assert 3 * 1024 * 1024 * 1365 < 2 ** 32 <= 3 * 1024 * 1024 * 1366
    assert _create(L, _grid((1024, 1024, 1365))) == 0
    assert _create(L, _grid((1024, 1024, 1366))) == E_ARG
    assert _create(L, _grid((1017, 1024, 1365))) == 0                  # px = 1024 as well
    assert _create(L, _grid((32, 32, 32), courant=0.5774)) == E_CFL     # S above 1/sqrt(3)


def test_batch_run_arguments_are_checked_on_the_host(L):
    """nlf_batch_run refuses a batch larger than NLF_MAX_BATCH (256) or
    without step counts before touching any context or the device, and an
    empty batch returns at once."""
    hs = (C.c_void_p * 257)()
    steps = (C.c_longlong * 257)()
    status = (C.c_int * 257)()
    assert L.nlf_batch_run(hs, 257, steps, None, status) == E_ARG
    assert L.nlf_batch_run(hs, 1, None, None, status) == E_ARG
    assert L.nlf_batch_run(hs, -1, steps, None, status) == E_ARG
    assert L.nlf_batch_run(hs, 0, steps, None, status) == 0          # an empty batch is no work
