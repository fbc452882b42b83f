"""Single-frequency plane maps (E and the free-electron charge density,
Sec. V / Eq. Nsol) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2005_06997_gb300 import nlfdtd
from paper_2005_06997_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("axis", [1, 2])
def test_plane_maps_match_oracle(axis):
    prob = W.small_sphere(n=36, steps=0, nf=8, K=4, band_ev=(1.5, 8.5))
    omega = np.array([3.0, 4.2, 5.5]) * W.EV_TO_RAD
    n3 = prob["shape"]
    idx = n3[axis] // 2
    prob["plane_map"] = {"axis": axis, "index": idx, "omega": omega, "K": prob["monitors"]["K"]}
    steps = 1200
    g = nlfdtd.Solver(prob)
    g.run(steps)
    g.sync()
    o = oracle.Sim(prob)
    o.set_plane(axis, idx, omega, prob["monitors"]["K"])
    o.step(steps)
    for q, name in enumerate(("Ex", "Ey", "Ez", "density")):
        got, want = g.plane_map(name), o.plane_dft(q)
        assert np.max(np.abs(want)) > 0, name
        assert rel_l2(got, want) <= 1e-4, (name, rel_l2(got, want))
    g.close()
    o.close()


def test_plane_monitor_rejected_in_batch():
    prob = W.small_sphere(n=36, steps=0, nf=4, K=4)
    prob["plane_map"] = {"axis": 2, "index": 18, "omega": [4.0 * W.EV_TO_RAD], "K": 4}
    s = nlfdtd.Solver(prob)
    assert nlfdtd.batch_run([s], [8]) == [-1]           # NLF_E_ARG
    s.close()
