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
"""
import ctypes as C
import os
import subprocess
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


def _build_stall_library(d):
    objs = []
    for src in build.sources():
        obj = os.path.join(d, os.path.basename(src) + ".o")
        subprocess.check_call([build.nvcc(), *build.ARCH, *build.FLAGS, "-DNLF_TEST_TMA_STALL=1", "-c", src,
                               "-o", obj])
        objs.append(obj)
    lib = os.path.join(d, "libnlfdtd_stall.so")
    subprocess.check_call([build.nvcc(), *build.ARCH, "-shared", "-o", lib, *objs])
    return lib


def test_tma_wait_that_runs_out_is_reported_and_the_device_stays_usable():
    with tempfile.TemporaryDirectory() as d:
        path = _build_stall_library(d)
        L = C.CDLL(path)
        for name, (res, args) in nlfdtd.SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
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
