"""The largest grid the C ABI accepts, on the GPU.

The kernels address the fields with 32-bit offsets; the library accepts a
grid while three components of a field fit them (3 px ny nz < 2^32, px = nx
rounded up to 8).  At that limit (1024 x 1024 x 1365 cells, 1.43 G cells,
69 GB of E and H) a divergence-free pulse placed in the far corner of the
grid, where the offsets are largest, must evolve as the same pulse does in
a small grid: in vacuum the update is the same at every cell, and both
pulses sit 80 cells from their nearest walls, which a front moving at most
half a cell per step (S = 0.5) does not reach in 100 steps, so the two
neighbourhoods agree to rounding."""
import numpy as np
import pytest
import torch

from paper_2005_06997_gb300 import nlfdtd
from paper_2005_06997_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEPS = 100
HALF = 60          # neighbourhood half-width compared (cells)
WIDTH = 5.0        # pulse 1/e half-width (cells)


def vacuum(n3):
    return {"shape": n3, "dx": 1e-9, "courant": 0.5, "pml": 0, "bc": ("pec",) * 3, "eps_b": 1.0,
            "materials": [], "shapes": [], "source": None, "monitors": None, "steps": 0}


def run(n3, centre):
    nx, ny, nz = n3
    ex, ey = W.curl_pulse((nz, ny, nx), centre, (WIDTH,) * 3)
    s = nlfdtd.Solver(vacuum(n3))
    s.set_field("Ex", ex)
    s.set_field("Ey", ey)
    del ex, ey
    s.run(STEPS)
    s.sync()
    ci, cj, ck = (int(round(c)) for c in centre)
    sl = (slice(ck - HALF, ck + HALF + 1), slice(cj - HALF, cj + HALF + 1), slice(ci - HALF, ci + HALF + 1))
    out = {}
    for f in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz"):
        out[f] = np.ascontiguousarray(s.field(f)[sl], dtype=np.float64)
    s.close()
    return out


def test_largest_grid_evolves_a_pulse_as_a_small_grid_does():
    free = torch.cuda.mem_get_info()[0]
    if free < 100 << 30:
        pytest.skip("needs about 80 GB of free device memory")
    big = (1024, 1024, 1365)
    assert 3 * big[0] * big[1] * big[2] < 2 ** 32
    far = (big[0] - 80, big[1] - 80, big[2] - 80)
    a = run(big, far)
    small = (160, 160, 160)
    b = run(small, (80, 80, 80))
    for vec in ("E", "H"):
        comps = [vec + c for c in "xyz"]
        num = sum(np.sum((a[c] - b[c]) ** 2) for c in comps)
        den = sum(np.sum(b[c] ** 2) for c in comps)
        assert den > 0
        print(vec, "relative L2 difference", np.sqrt(num / den))
        assert np.sqrt(num / den) <= 1e-6, (vec, np.sqrt(num / den))
