"""Pins of the oracle's single-frequency plane maps (E and the free-electron
charge density div P_f of Sec. V, Eq. Nsol), independent of the CUDA path.

* The density operator against the closed form of the discrete divergence of
  analytic P fields (periodic axes) and against the PEC edge (P_f = 0 outside
  the grid).
* The plane DFT of E_x in the total-field region of a vacuum run against the
  flux monitors' incident record, a separate code path over the 1D grid: the
  TF/SF connection reproduces the incident wave exactly there.
* The accumulation (plane slicing, phase, rectangle-rule scale) against a
  DFT taken here from per-step snapshots, for every plane axis.
"""
import copy

import numpy as np
import pytest

import oracle
from paper_2005_06997_gb300 import workloads as W


def periodic_problem(n3, dx):
    return {"shape": tuple(n3), "dx": dx, "courant": 0.5, "pml": 0, "bc": ("periodic",) * 3,
            "materials": [], "shapes": [], "source": None, "monitors": None}


def test_density_matches_discrete_divergence_closed_form():
    n3, dx = (16, 12, 10), 0.5e-9
    sim = oracle.Sim(periodic_problem(n3, dx))
    nz, ny, nx = sim.shape3
    k1, k2 = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    A, B = 2.0e-3, -0.7e-3
    # P_x at the E_x site (i + 1/2) dx, P_y at (j + 1/2) dx
    sim.array("Px")[...] = A * np.cos(k1 * (i + 0.5)) * np.ones((nz, ny, 1))
    sim.array("Py")[...] = B * np.cos(k2 * (j + 0.5)) * np.ones((nz, 1, nx))
    d = sim.density()
    want = (-2 * A / dx * np.sin(k1 / 2) * np.sin(k1 * i)) + (-2 * B / dx * np.sin(k2 / 2) * np.sin(k2 * j))
    assert np.max(np.abs(d - want)) <= 1e-12 * np.max(np.abs(want))


def test_density_at_a_pec_wall_sees_zero_beyond_it():
    prob = periodic_problem((8, 8, 8), 1e-9)
    prob["bc"] = ("periodic", "periodic", "pec")
    sim = oracle.Sim(prob)
    C = 3.0e-3
    sim.array("Pz")[...] = C
    d = sim.density()
    assert np.allclose(d[0], C / 1e-9, rtol=1e-14)          # P_z(k - 1) = 0 below the grid
    assert np.max(np.abs(d[1:])) == 0.0


def test_vacuum_plane_map_in_total_field_equals_incident_record():
    prob = W.small_sphere(n=36, steps=0, nf=6, K=4, band_ev=(1.5, 8.5))
    prob["shapes"] = []
    src, mon = prob["source"], prob["monitors"]
    kc = (mon["abs_lo"][2] + mon["abs_hi"][2]) // 2
    sim = oracle.Sim(prob)
    sim.set_plane(2, kc, mon["omega"], mon["K"])
    sim.step(600)
    Ex = sim.plane_dft(0)                                  # [nf][ny][nx]
    aE, _ = sim.dft()
    inc = aE[-1, :, 0] + 1j * aE[-1, :, 1]                 # the incident record, same K dt scale
    lo, hi = src["tf_lo"], src["tf_hi"]
    tf = Ex[:, lo[1]:hi[1] + 1, lo[0]:hi[0]]
    assert np.max(np.abs(tf - inc[:, None, None])) <= 1e-10 * np.max(np.abs(inc))
    sf = Ex.copy()
    sf[:, lo[1]:hi[1] + 1, lo[0]:hi[0]] = 0
    assert np.max(np.abs(sf)) <= 1e-10 * np.max(np.abs(inc))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_plane_accumulation_matches_snapshot_dft(axis):
    prob = W.small_sphere(n=30, radius_cells=4.0, pml=4, steps=0, nf=4, K=1, band_ev=(2.0, 6.0))
    prob["monitors"] = None
    omega = np.array([3.0, 4.5, 5.2]) * W.EV_TO_RAD
    idx = 15 if axis != 2 else 14
    sim = oracle.Sim(prob)
    sim.set_plane(axis, idx, omega, 3)
    dt = sim.dt
    want = {q: 0.0 for q in range(4)}
    names = ("Ex", "Ey", "Ez")
    for n in range(1, 61):
        sim.step(1)
        if n % 3:
            continue
        d = sim.density()
        snaps = [np.take(sim.array(c), idx, axis=2 - axis) for c in names] + [np.take(d, idx, axis=2 - axis)]
        ph = np.exp(1j * omega * n * dt) * 3 * dt
        for q in range(4):
            want[q] = want[q] + ph[:, None, None] * snaps[q][None]
    for q in range(4):
        got = sim.plane_dft(q)
        scale = np.max(np.abs(want[q]))
        assert scale > 0
        assert np.max(np.abs(got - want[q])) <= 1e-12 * scale, q
