"""Failure detection on the GPU without faulting it.

* The whole-grid watchdog: a context without flux monitors (so no flux-face
  samples to watch) whose field is poisoned with one NaN on the host reports
  NLF_E_UNSTABLE at its next sync.
* The bounded mbarrier wait: a test-only build of the library (compiled here
  with NLF_TEST_TMA_STALL) makes the first E stage of every background-tile
  block expect 16 bytes more than its copy delivers.  The copy lands in full
  (nothing is left in flight), the stage's barrier never completes, the
  shortened bounded wait gives up, the block leaves after waiting (bounded)
  for its other copies, and nlf_sync reports NLF_E_CUDA with the
  tensor-memory message.  The device stays usable: the product library then
  runs a normal solve.
* The bounds-checked build (NLF_BOUNDS_CHECK): every non-TMA global access
  of the kernels is checked against its array's extent; a violation skips
  the access and is recorded for nlf_sync.  Clean runs record nothing and
  give the product's results.
"""
import ctypes as C
import os
import tempfile

import numpy as np
import pytest

from paper_2005_06997_gb300 import build, nlfdtd
from paper_2005_06997_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_whole_grid_watchdog_reports_a_poisoned_field():
    prob = W.small_sphere(n=40, steps=0, nf=8, K=4)
    prob["monitors"] = None
    s = nlfdtd.Solver(prob)
    s.run(0)
    ex = np.zeros(s.shape3, dtype=np.float32)
    ex[20, 5, 30] = np.nan                       # far from the sphere and the TF surface
    s.set_field("Ex", ex)
    s.run(512)
    with pytest.raises(nlfdtd.NLFError) as e:
        s.sync()
    assert e.value.code == -6
    s.close()


def _build_library(d, define, name):
    """A variant of the library compiled with `define`, loaded with the same
    signatures as the product's."""
    path = build.build(extra=[define], lib=os.path.join(d, name))
    L = C.CDLL(path)
    for fname, (res, args) in nlfdtd.SIGNATURES.items():
        fn = getattr(L, fname)
        fn.restype = res
        fn.argtypes = args
    return L


def test_tma_wait_that_runs_out_is_reported_and_the_device_stays_usable():
    with tempfile.TemporaryDirectory() as d:
        L = _build_library(d, "-DNLF_TEST_TMA_STALL=1", "libnlfdtd_stall.so")
        # a vacuum grid with PEC walls: every tile is a background tile
        prob = {"shape": (64, 48, 40), "dx": 1e-9, "courant": 0.5, "pml": 0, "bc": ("pec",) * 3, "eps_b": 1.0,
                "materials": [], "shapes": [], "source": None, "monitors": None}
        h = C.c_void_p()
        g = nlfdtd.make_grid(prob)
        assert L.nlf_create(C.byref(g), C.byref(h)) == 0
        assert L.nlf_run(h, 4, None) == 0
        rc = L.nlf_sync(h, 60000)
        msg = L.nlf_last_error(h)
        L.nlf_destroy(h)
    assert rc == -5, (rc, msg)
    assert b"tensor-memory copy" in msg
    # the product library on the same device afterwards
    s = nlfdtd.Solver(W.small_sphere(n=36, steps=0, nf=8, K=4))
    s.run(64)
    s.sync()
    assert np.all(np.isfinite(s.field("Ex")))
    s.close()


# ------------------------------------------------- bounds-checked build

def _context(L, prob):
    h = C.c_void_p()
    g = nlfdtd.make_grid(prob)
    assert L.nlf_create(C.byref(g), C.byref(h)) == 0
    mats, nm = nlfdtd.make_materials(prob)
    assert L.nlf_set_materials(h, mats, nm) == 0
    shp, ns = nlfdtd.make_shapes(prob)
    assert L.nlf_set_shapes(h, shp, ns) == 0
    keep = []
    if prob.get("source") is not None:
        src = nlfdtd.make_source(prob["source"])
        assert L.nlf_set_source(h, C.byref(src)) == 0
    if prob.get("monitors") is not None:
        mon, om = nlfdtd.make_monitors(prob["monitors"])
        keep.append(om)
        assert L.nlf_set_monitors(h, C.byref(mon)) == 0
    return h, keep


def _field(L, h, prob, name):
    out = np.empty(tuple(reversed(prob["shape"])), dtype=np.float32)
    assert L.nlf_get_field(h, nlfdtd.FIELD[name], out.ctypes.data, 0) == 0
    return out


def _problems():
    sphere = W.small_sphere(n=36, steps=0, nf=8, K=4)
    fused = W.small_sphere(n=80, radius_cells=23.0, pml=6, material=W.AU_LIKE_GNOR, steps=0, nf=8, K=4,
                           center_offset_half=(0, 0, 0))
    return [("sphere", sphere, 300), ("fused_tiles", fused, 200)]


def test_bounds_checked_build_runs_clean_and_matches():
    """The -DNLF_BOUNDS_CHECK build checks every non-TMA global access of
    the step, material, TF/SF and DFT kernels against its array's size:
    single grids with site-list and fused material updates, and a batch of
    uneven grids, record no violation and give the product's results."""
    with tempfile.TemporaryDirectory() as d:
        L = _build_library(d, "-DNLF_BOUNDS_CHECK=1", "libnlfdtd_checked.so")
        for tag, prob, steps in _problems():
            h, keep = _context(L, prob)
            assert L.nlf_run(h, steps, None) == 0
            rc = L.nlf_sync(h, -1)
            assert rc == 0, (tag, L.nlf_last_error(h))
            ref = nlfdtd.Solver(prob)
            ref.run(steps)
            ref.sync()
            for f in ("Ex", "Hy", "Px"):
                a, b = _field(L, h, prob, f), ref.field(f)
                assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b), (tag, f)
            ref.close()
            L.nlf_destroy(h)
        # a batch of uneven grids through the batched kernels
        probs = W.batched_instances(n=4, nf=16, steps=0)
        hs = [_context(L, q) for q in probs]
        arr = (C.c_void_p * len(hs))(*[x[0].value for x in hs])
        steps = (C.c_longlong * len(hs))(*([600] * len(hs)))
        status = (C.c_int * len(hs))()
        L.nlf_batch_run(arr, len(hs), steps, None, status)
        assert list(status) == [0] * len(hs)
        for (h, _), q in zip(hs, probs):
            rc = L.nlf_sync(h, -1)
            assert rc == 0, L.nlf_last_error(h)
            L.nlf_destroy(h)
