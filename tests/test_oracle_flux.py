"""Pin of the oracle's flux-box assembly by Poynting's theorem.

The absorption cross section of Sec. V is read as the net inward flux of the
time-averaged Poynting vector through a closed box around the particle,
assembled from running DFTs of the face fields (E at n dt, H averaged over
the two half cells around the face at (n - 1/2) dt, trapezoid weights on the
face edges, outward signs).  Poynting's theorem fixes that same power
independently, from the particle's interior: with fields varying as
exp(-i w t) the power the polarisation current J = dP/dt delivers to the
metal is (1/2) Re(J . E*) = (1/2) w Im(P E*) per unit volume.  Summed over
the metal's E-sites (each of volume dx^3) from DFTs of P_f and E taken here,
in this file, from the oracle's arrays every K steps, and divided by the
incident intensity, it must equal the flux-box sigma_abs.  Nothing here
re-uses the face records: a wrong edge weight, an H sample one cell off, a
flipped face or term sign, or a wrong half-step phase breaks the equality.

A Drude sphere with a large damping rate lets the fields decay before the
run ends, so both DFTs see complete signals.
"""
import math

import numpy as np

import oracle
from paper_2005_06997_gb300 import workloads as W


def absorption_two_ways(gamma_ev=1.2, nf=16, K=8, after_gamma=14.0):
    mat = W.drude_material(9.0, gamma_ev)
    prob = W.small_sphere(n=30, pml=5, radius_cells=3.5, steps=0, band_ev=(2.5, 8.5), nf=nf, K=K, dx=1e-9,
                          material=mat, center_offset_half=(0, 0, 0))
    sim = oracle.Sim(prob)
    w = np.asarray(prob["monitors"]["omega"])
    vox = sim.material_map()
    sites = [np.flatnonzero(vox[c].reshape(-1)) for c in range(3)]
    steps = int((prob["source"]["t0"] + after_gamma / mat["gamma"]) / sim.dt) // K * K
    accE = [np.zeros((len(s), nf), complex) for s in sites]
    accP = [np.zeros((len(s), nf), complex) for s in sites]
    for _ in range(steps // K):
        sim.step(K)
        ph = np.exp(1j * w * sim.n * sim.dt) * K * sim.dt
        for c, nm in enumerate("xyz"):
            e = np.asarray(sim.array("E" + nm)).reshape(-1)[sites[c]]
            p = np.asarray(sim.array("P" + nm)).reshape(-1)[sites[c]]
            accE[c] += e[:, None] * ph[None, :]
            accP[c] += p[:, None] * ph[None, :]
    sp = sim.spectra()
    dV = prob["dx"] ** 3
    power = sum(0.5 * w[None, :] * np.imag(accP[c] * np.conj(accE[c])) for c in range(3)).sum(axis=0) * dV
    return w, sp, power / sp["inc"]


def test_flux_box_absorption_equals_volume_absorption():
    w, sp, s_vol = absorption_two_ways()
    peak = np.max(s_vol)
    assert peak > 0
    # measured agreement ~2e-4 of the peak; the bound leaves a factor of ten
    assert np.max(np.abs(sp["abs"] - s_vol)) <= 2e-3 * peak
    # and the line is really there: the volume absorption has a resonance
    assert np.argmax(s_vol) not in (0, len(w) - 1)
