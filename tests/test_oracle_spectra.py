"""Pins of the oracle's running DFT, flux boxes and cross-section normalisation.

* The DFT of the incident field at the centre plane must reproduce the
  analytic Fourier transform of the Gaussian-modulated source (magnitude),
  and I(w) = Re(E H*)/2 must equal |E|^2/(2 eta0) for a plane wave.
* A small Drude sphere must reproduce quasi-static Mie theory (Sec. V compares
  against Mie theory): the integrated absorption of
  sigma_abs = k Im(alpha), alpha = 4 pi R^3 (eps-1)/(eps+2), R from the voxel
  count, and the resonance near eps(w) = -2.  A staircased sphere of R = 4
  cells resonates a few per cent low (5.8 % at R = 4, 1.9 % at R = 8 cells:
  first order in dx/R) and its line is broadened, so the pin is the area and
  the position, not the peak height.  sigma_sca >= 0 and small; the nonlocal
  resonance is blue-shifted with respect to the local one (Sec. V).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_06997_gb300 import workloads as W

EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6
C0 = 1.0 / math.sqrt(EPS0 * MU0)
ETA0 = math.sqrt(MU0 / EPS0)


def gaussian_ft_mag(w, src):
    """|int f(t) exp(i w t) dt| for f = A exp(-((t-t0)/tau)^2) sin(w0 (t-t0))."""
    tau, w0, A = src["tau"], src["w0"], src["amp"]
    g = lambda x: math.sqrt(math.pi) * tau * np.exp(-(x * tau / 2) ** 2)
    return A * np.abs(g(w - w0) - g(w + w0)) / 2


def test_incident_spectrum_and_intensity():
    prob = W.small_sphere(n=32, pml=5, radius_cells=4.0, steps=0, band_ev=(2.0, 8.0), nf=12, K=4, dx=1e-9,
                          material=W.drude_material(9.0, 0.5))
    prob["shapes"] = []
    sim = oracle.Sim(prob)
    # let the whole pulse pass the centre plane
    src = prob["source"]
    steps = int((src["t0"] + 5 * src["tau"]) / sim.dt) + 200
    sim.step(steps)
    aE, aH = sim.dft()
    Einc = aE[-1, :, 0] + 1j * aE[-1, :, 1]
    Hinc = aH[-1, :, 0] + 1j * aH[-1, :, 1]
    w = prob["monitors"]["omega"]
    ref = gaussian_ft_mag(w, src)
    sel = ref > 0.05 * ref.max()
    assert np.all(np.abs(np.abs(Einc[sel]) / ref[sel] - 1) < 0.01)
    I = sim.spectra()["inc"]
    assert np.all(np.abs(I[sel] / (np.abs(Einc[sel]) ** 2 / (2 * ETA0)) - 1) < 0.01)
    # no scatterer: both cross-sections vanish (up to the truncated pulse tail)
    sp = sim.spectra()
    area = (prob["shape"][0] * prob["dx"]) ** 2
    assert np.max(np.abs(sp["ext"][sel])) < 1e-6 * area


def run_sphere(beta):
    mat = W.drude_material(9.0, 0.5, beta=beta)
    prob = W.small_sphere(n=32, pml=5, radius_cells=4.0, steps=0, band_ev=(2.0, 9.0), nf=141, K=8, dx=1e-9,
                          material=mat, center_offset_half=(0, 0, 0))
    sim = oracle.Sim(prob)
    g = mat["gamma"]
    steps = int((prob["source"]["t0"] + 16.0 / g) / sim.dt)
    sim.step(steps)
    return prob, sim


@pytest.mark.slow
def test_small_drude_sphere_matches_quasistatic_mie():
    prob, sim = run_sphere(0.0)
    sp = sim.spectra()
    w = prob["monitors"]["omega"]
    mat = prob["materials"][0]
    nsites = np.count_nonzero(sim.material_map()[0])
    R = (3 * nsites / (4 * math.pi)) ** (1 / 3) * prob["dx"]
    eps = 1 - mat["wp"] ** 2 / (w ** 2 + 1j * mat["gamma"] * w)
    alpha = 4 * math.pi * R ** 3 * (eps - 1) / (eps + 2)
    s_abs_mie = (w / C0) * alpha.imag
    i_fd, i_mie = np.argmax(sp["abs"]), np.argmax(s_abs_mie)
    assert abs(w[i_fd] / w[i_mie] - 1) < 0.07
    assert abs(np.trapezoid(sp["abs"], w) / np.trapezoid(s_abs_mie, w) - 1) < 0.05
    assert np.all(sp["sca"] > -1e-3 * sp["abs"].max())
    assert sp["sca"].max() < 0.05 * sp["abs"].max()
    assert np.allclose(sp["ext"], sp["abs"] + sp["sca"])
    # nonlocal pressure term: resonance moves to higher frequency
    prob_nl, sim_nl = run_sphere(1.07e6 * 4)
    w_nl = w[np.argmax(sim_nl.spectra()["abs"])]
    assert w_nl > w[i_fd]
