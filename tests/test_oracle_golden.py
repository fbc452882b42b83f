"""Pins of the oracle against values the paper prints (fixtures in tests/golden/).

* The raised-cosine pulse of Sec. V (SI movies paragraph): the paper gives
  f(t) = [(1 - cos(w_max t)) / 2]^3 with w_max = 1.26e16 rad/s, and the
  wavelength 150 nm for that frequency.  The oracle's hard source must follow
  the pulse written as its finite cosine series (an algebraically different
  form: 5/16 - 15/32 cos x + 3/16 cos 2x - 1/32 cos 3x on one period, zero
  after), and the running DFT of the incident wave at the centre plane must
  reproduce the pulse's Fourier integral over that period in closed form.
* The EELS comparison of Sec. V puts the spheres in a background of index
  n = 1.3: in that background the incident intensity the flux normalisation
  divides by must be n |E|^2 / (2 eta0), the plane-wave relation.
* The silver set-up of Sec. V: beta^2 = v_F^2 / 3 with v_F = 1.39e6 m/s and
  a cell of D/100; the hydrodynamic stability bound of the discrete scheme
  (beta dt sqrt(3) / dx <= 1) holds there with a wide margin, and the cell
  stays below the quoted Fermi wavelength.
"""
import math
import os

import numpy as np

import oracle
from paper_2005_06997_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6
C0 = 1.0 / math.sqrt(EPS0 * MU0)
ETA0 = math.sqrt(MU0 / EPS0)

# [(1 - cos x)/2]^3 expanded into cosines of x, 2x, 3x
SERIES = (5.0 / 16.0, -15.0 / 32.0, 3.0 / 16.0, -1.0 / 32.0)


def golden(name):
    """key = value lines of a fixture ('#' starts a comment); several values
    on one line give a tuple."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (s.strip() for s in line.split("=", 1))
            vals = tuple(float(v) for v in val.split())
            out[key] = vals[0] if len(vals) == 1 else vals
    return out


def pulse_series(t, w_max):
    x = w_max * np.asarray(t, dtype=np.float64)
    f = sum(a * np.cos(m * x) for m, a in enumerate(SERIES))
    return np.where((x >= 0) & (x <= 2 * math.pi), f, 0.0)


def pulse_fourier(w, w_max):
    """int_0^T f(t) exp(i w t) dt over the one period T = 2 pi / w_max, from
    int_0^T cos(m W t) exp(i w t) dt = (exp(i w T) - 1)/i * w / (w^2 - m^2 W^2)."""
    T = 2 * math.pi / w_max
    w = np.asarray(w, dtype=np.float64)
    s = sum(a * w / (w ** 2 - (m * w_max) ** 2) for m, a in enumerate(SERIES))
    return (np.exp(1j * w * T) - 1.0) / 1j * s


def raised_cos_problem(n_background=1.0, nf=24, band_ev=(0.5, 8.0), K=4):
    g = golden("raised_cosine_source.txt")
    prob = W.small_sphere(n=32, pml=5, radius_cells=4.0, steps=0, band_ev=band_ev, nf=nf, K=K, dx=1e-9,
                          material=W.drude_material(9.0, 0.5))
    prob["shapes"] = []
    prob["eps_b"] = n_background ** 2
    src = prob["source"]
    prob["source"] = W.raised_cos_source(src["tf_lo"], src["tf_hi"], w_max=g["w_max_rad_s"])
    return prob, g


def test_printed_w_max_matches_printed_wavelength():
    g = golden("raised_cosine_source.txt")
    assert g["exponent"] == 3
    w_from_lambda = 2 * math.pi * C0 / g["lambda_of_w_max_m"]
    # the paper rounds to three significant figures
    assert abs(w_from_lambda / g["w_max_rad_s"] - 1) < 5e-3


def test_hard_source_follows_the_printed_raised_cosine():
    prob, g = raised_cos_problem()
    w_max = g["w_max_rad_s"]
    sim = oracle.Sim(prob)
    dt = sim.dt
    period_steps = int(2 * math.pi / w_max / dt) + 1
    got, t = [], []
    for _ in range(period_steps + 20):
        sim.step(1)
        e, _, _ = sim.inc()
        got.append(e[0])
        t.append(sim.n * dt)
    got, t = np.array(got), np.array(t)
    ref = pulse_series(t, w_max)
    assert np.max(np.abs(got - ref)) < 1e-14
    # the pulse peaks at 1 half-way through its period and is zero after it
    assert abs(np.max(got) - 1.0) < 1e-3
    assert np.all(got[t > 2 * math.pi / w_max] == 0.0)


def test_raised_cosine_incident_spectrum_in_the_n13_background():
    n_b = golden("silver_sphere_setup.txt")["background_index"]
    for n in (1.0, n_b):
        prob, g = raised_cos_problem(n_background=n)
        w_max = g["w_max_rad_s"]
        sim = oracle.Sim(prob)
        # the whole pulse has passed the centre plane well before this
        sim.step(int(2 * math.pi / w_max / sim.dt) + 40 * 2 * 16)
        aE, aH = sim.dft()
        Einc = aE[-1, :, 0] + 1j * aE[-1, :, 1]
        w = prob["monitors"]["omega"]
        ref = np.abs(pulse_fourier(w, w_max))
        sel = ref > 0.05 * ref.max()
        assert np.count_nonzero(sel) >= 10
        assert np.all(np.abs(np.abs(Einc[sel]) / ref[sel] - 1) < 0.01), (n, np.abs(Einc[sel]) / ref[sel])
        # plane wave in index n: H = n E / eta0, so I = n |E|^2 / (2 eta0)
        I = sim.spectra()["inc"]
        assert np.all(np.abs(I[sel] / (n * np.abs(Einc[sel]) ** 2 / (2 * ETA0)) - 1) < 0.01)
        # no scatterer: nothing crosses the flux boxes
        area = (prob["shape"][0] * prob["dx"]) ** 2
        assert np.max(np.abs(sim.spectra()["ext"][sel])) < 1e-6 * area


def test_silver_setup_is_inside_the_discrete_stability_bounds():
    s = golden("silver_sphere_setup.txt")
    beta = math.sqrt(s["beta_squared_over_vF_squared"]) * s["fermi_velocity_m_s"]
    assert abs(beta - 1.39e6 / math.sqrt(3)) < 1.0
    prob = W.small_sphere(n=32, pml=5, radius_cells=4.0, steps=0, nf=4, K=4)
    for D in s["diameters_m"]:
        dx = D / s["cells_per_diameter"]
        # the paper's reason for D/100: the cell is below the Fermi wavelength
        assert dx < s["fermi_wavelength_m"]
        prob["dx"] = dx
        prob["materials"] = [W.drude_material(9.0, 0.02, beta=beta)]
        sim = oracle.Sim(prob)
        assert abs(sim.dt - 0.5 * dx / C0) < 1e-12 * sim.dt
        # hydrodynamic bound of the longitudinal mode: beta dt sqrt(3) / dx <= 1
        assert beta * sim.dt * math.sqrt(3) / dx < 1e-2
