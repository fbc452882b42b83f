"""The z chunks of the EM z-march, checked on the host: a small program
built from nlf_internal.h (the same inline functions the kernels and the
site-list classification call) walks every grid depth, CPML width and chunk
length in a range (tests/native/zchunk_check.cu)."""
import os
import subprocess
import tempfile

import pytest

from paper_2005_06997_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_z_chunks_tile_the_grid_and_keep_interior_chunks_clear_of_the_slabs():
    try:
        nvcc = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "zchunk_check")
        subprocess.check_call([nvcc, "-std=c++17", "-I" + build.CSRC, "-I" + build.INCLUDE,
                               os.path.join(HERE, "native", "zchunk_check.cu"), "-o", exe])
        r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 failures" in r.stdout
