"""Seeded synthetic problem descriptions (inputs only, no FDTD arithmetic).

Both the CUDA path and the CPU oracle consume these plain dicts; this module
holds none of the method's arithmetic.  It only places geometry on the grid,
converts physical sizes to integer half-cell units (round half to even) and
converts eV to rad/s.

A problem dict has the keys
  shape (nx, ny, nz), dx [m], courant, pml, bc (3 x 'pec'|'cpml'|'periodic'),
  eps_b, materials [ {eps_inf, wp, gamma, beta, diff, poles=[(A, Om, Ga, phi)]} ],
  shapes [ {kind, material (1-based), c (half cells), radius | half | side, tip_*} ],
  source {tf_lo, tf_hi, waveform, w0, tau, t0, amp} or None,
  monitors {omega [rad/s], abs_lo, abs_hi, sca_lo, sca_hi, K} or None,
  steps.

The workloads mirror the paper's scales (sub-nanometre cells and a few-nm
metal spheres, Sec. V; a larger particle with sharp extrusions, Sec. VI).  The
paper's silver critical-points fit, its Mie codes and its measured data are not
available, so the materials are Drude-like with the stated hydrodynamic
parameters and one Lorentz pole where a bound-electron response is asked for.
"""
from __future__ import annotations

import math

import numpy as np

EV = 1.602176634e-19          # J
HBAR = 1.054571817e-34        # J s
EV_TO_RAD = EV / HBAR         # rad/s per eV
C0 = 299792458.0              # m/s

PML_MARGIN_TF = 4             # TF box inset from the CPML (cells)
SCA_OUTSET = 2                # scattering box outside the TF box (cells)
ABS_MARGIN = 2                # absorption box around the particle (cells)
METAL_MARGIN = 2              # metal at least this far inside the TF box (cells)


def ev(x):
    return np.asarray(x, dtype=np.float64) * EV_TO_RAD if np.ndim(x) else float(x) * EV_TO_RAD


def half_cells(length_m: float, dx: float) -> int:
    """A physical length in integer half-cell units (round half to even)."""
    return int(np.rint(length_m / (0.5 * dx)))


# ---------------------------------------------------------------- materials

def drude_material(wp_ev, gamma_ev, beta=0.0, diff=0.0, eps_inf=1.0, poles=()):
    return {"eps_inf": eps_inf, "wp": ev(wp_ev), "gamma": ev(gamma_ev), "beta": beta, "diff": diff,
            "poles": [tuple(p) for p in poles]}


def lorentz_pole(A=1.0, omega_ev=4.0, gamma_ev=0.4, phi=0.0):
    return (A, ev(omega_ev), ev(gamma_ev), phi)


AG_LIKE = drude_material(9.0, 0.02, beta=1.07e6, diff=0.0)
AU_LIKE_GNOR = drude_material(9.0, 0.07, beta=1.2e6, diff=1.9e-4, poles=[lorentz_pole()])


# ------------------------------------------------------------------ sources

def gaussian_source(tf_lo, tf_hi, band_ev, amp=1.0):
    """Gaussian-modulated sine whose amplitude spectrum falls to 1/e at the band edges."""
    lo, hi = band_ev
    w0 = ev(0.5 * (lo + hi))
    half_band = ev(0.5 * (hi - lo))
    tau = 2.0 / half_band
    return {"tf_lo": tuple(tf_lo), "tf_hi": tuple(tf_hi), "waveform": "gaussian",
            "w0": w0, "tau": tau, "t0": 4.0 * tau, "amp": amp}


def raised_cos_source(tf_lo, tf_hi, w_max=1.26e16, amp=1.0):
    return {"tf_lo": tuple(tf_lo), "tf_hi": tuple(tf_hi), "waveform": "raised_cos",
            "w0": w_max, "tau": 0.0, "t0": 0.0, "amp": amp}


# ----------------------------------------------------------------- problems

def _boxes(n3, pml, ext_lo, ext_hi):
    """TF, absorption and scattering boxes (node indices) for a particle
    whose E-sites lie inside cells [ext_lo, ext_hi]."""
    tf_lo = tuple(pml + PML_MARGIN_TF for _ in range(3))
    tf_hi = tuple(n - pml - PML_MARGIN_TF for n in n3)
    # the absorption box keeps one cell inside the TF box so that both H samples
    # averaged onto each of its faces are total fields
    abs_lo = tuple(max(int(e) - ABS_MARGIN, t + 1) for e, t in zip(ext_lo, tf_lo))
    abs_hi = tuple(min(int(e) + ABS_MARGIN, t - 1) for e, t in zip(ext_hi, tf_hi))
    sca_lo = tuple(t - SCA_OUTSET for t in tf_lo)
    sca_hi = tuple(t + SCA_OUTSET for t in tf_hi)
    for a in range(3):
        if ext_lo[a] < tf_lo[a] + METAL_MARGIN or ext_hi[a] > tf_hi[a] - METAL_MARGIN:
            raise ValueError("particle does not fit inside the TF box with the metal margin")
    return tf_lo, tf_hi, abs_lo, abs_hi, sca_lo, sca_hi


def _extent_cells(c_half, r_half):
    lo = [math.floor((c - r) / 2) for c, r in zip(c_half, r_half)]
    hi = [math.ceil((c + r) / 2) for c, r in zip(c_half, r_half)]
    return lo, hi


def scatter_problem(n3, dx, pml, materials, shapes, extent_half, steps, band_ev, nf=200, K=16,
                    courant=0.5, eps_b=1.0):
    """Generic particle-in-a-box problem: CPML on every axis, TF/SF source
    along +z polarised along x, absorption and scattering flux boxes."""
    c_half, r_half = extent_half
    ext_lo, ext_hi = _extent_cells(c_half, r_half)
    tf_lo, tf_hi, abs_lo, abs_hi, sca_lo, sca_hi = _boxes(n3, pml, ext_lo, ext_hi)
    omega = ev(np.linspace(band_ev[0], band_ev[1], nf))
    return {
        "shape": tuple(n3), "dx": dx, "courant": courant, "pml": pml, "bc": ("cpml",) * 3,
        "eps_b": eps_b, "materials": materials, "shapes": shapes,
        "source": gaussian_source(tf_lo, tf_hi, band_ev),
        "monitors": {"omega": omega, "abs_lo": abs_lo, "abs_hi": abs_hi, "sca_lo": sca_lo,
                     "sca_hi": sca_hi, "K": K},
        "steps": steps,
    }


def sphere_shape(center_half, radius_half, material=1):
    return {"kind": "sphere", "material": material, "c": tuple(int(c) for c in center_half),
            "radius": int(radius_half)}


def sphere_problem(n, dx, radius_m, pml, material, steps, band_ev=(2.0, 6.0), nf=200, K=16,
                   courant=0.5, center_offset_half=(0, 0, 0)):
    R = half_cells(radius_m, dx)
    c = tuple(n + o for o in center_offset_half)        # grid centre = node n/2 = half-cell n
    sh = [sphere_shape(c, R)]
    return scatter_problem((n, n, n), dx, pml, [material], sh, (c, (R, R, R)), steps, band_ev, nf, K,
                           courant)


def cube_tips_shape(center_half, side_m, tip_base_m, tip_height_m, tip_radius_m, dx, material=1):
    """Cube with a rounded square pyramid on each face centre (integer half cells)."""
    a = 2 * (half_cells(side_m, dx) // 2)
    b = 2 * (half_cells(tip_base_m, dx) // 2)
    h = half_cells(tip_height_m, dx)
    r = half_cells(tip_radius_m, dx)
    A, B = a // 2, b // 2
    slant = math.sqrt(B * B + h * h)
    x0 = A + h - r * slant / B            # rounding sphere tangent to the four faces
    cut = x0 + r * B / slant              # plane of the tangency circle
    return {"kind": "cube_tips", "material": material, "c": tuple(int(c) for c in center_half),
            "side": a, "tip_base": b, "tip_height": h, "tip_radius": r,
            "tip_center": int(np.rint(x0)), "tip_cut": int(np.rint(cut))}


# ------------------------------------------------------------ named configs

def config_sphere_ag_48():
    """Ag-like sphere r = 2 nm, 48^3 cells at 0.25 nm with an 8-cell CPML, Courant 0.5,
    nonlocal Drude (D = 0), 2-6 eV, 1000 steps, 200 frequencies."""
    return sphere_problem(48, 0.25e-9, 2e-9, 8, AG_LIKE, 1000, (2.0, 6.0))


def config_sphere_au_gnor_224():
    """Au-like GNOR sphere r = 10 nm with a Lorentz pole, 224^3 cells at 0.2 nm,
    12-cell CPML, 8000 steps, 2-6 eV, 200 frequencies."""
    return sphere_problem(224, 0.2e-9, 10e-9, 12, AU_LIKE_GNOR, 8000, (2.0, 6.0))


def config_cube_tips_512():
    """60 nm Au-like cube with six rounded pyramidal tips (3 nm apex radius), GNOR,
    512^3 cells at 0.25 nm, 12-cell CPML, 10000 steps, 1-5 eV."""
    n, dx = 512, 0.25e-9
    sh = cube_tips_shape((n, n, n), 60e-9, 12e-9, 10e-9, 3e-9, dx)
    reach = sh["side"] // 2 + sh["tip_height"]
    return scatter_problem((n, n, n), dx, 12, [AU_LIKE_GNOR], [sh], ((n, n, n), (reach,) * 3),
                           10000, (1.0, 5.0))


def config_cube_tips_256():
    """The 512^3 cube with tips at half size in every length (30 nm cube, tips
    of 6 nm base, 5 nm height, 1.5 nm apex radius, 256^3 cells at 0.25 nm,
    12-cell CPML, 5000 steps, 1-5 eV): the same kernels on a state of a few
    GB, for profiler captures."""
    n, dx = 256, 0.25e-9
    sh = cube_tips_shape((n, n, n), 30e-9, 6e-9, 5e-9, 1.5e-9, dx)
    reach = sh["side"] // 2 + sh["tip_height"]
    return scatter_problem((n, n, n), dx, 12, [AU_LIKE_GNOR], [sh], ((n, n, n), (reach,) * 3),
                           5000, (1.0, 5.0))


CONFIGS = {
    "sphere_ag_r2nm_48": config_sphere_ag_48,
    "sphere_au_gnor_r10nm_224": config_sphere_au_gnor_224,
    "cube_tips_au_gnor_512": config_cube_tips_512,
    "cube_tips_au_gnor_256": config_cube_tips_256,
}


def curl_pulse(shape3, center, width):
    """A divergence-free initial E on the Yee lattice: the discrete curl of
    A z-hat, A a separable Gaussian (centre and 1/e half-widths in cells, x,
    y, z) held at the (i+1/2, j+1/2, k) points, so that E_x[k, j, i] = A[k,
    j, i] - A[k, j-1, i] and E_y[k, j, i] = A[k, j, i-1] - A[k, j, i]; the
    tangential E on the walls is zero.  Returns (E_x, E_y) as [nz][ny][nx]
    float32 arrays (unit peak of A)."""
    nz, ny, nx = shape3
    gx = np.exp(-(((np.arange(nx) + 0.5 - center[0]) / width[0]) ** 2)).astype(np.float32)
    gy = np.exp(-(((np.arange(ny) + 0.5 - center[1]) / width[1]) ** 2)).astype(np.float32)
    gz = np.exp(-(((np.arange(nz) - center[2]) / width[2]) ** 2)).astype(np.float32)
    dy = np.zeros(ny, np.float32)
    dy[1:] = gy[1:] - gy[:-1]
    dx = np.zeros(nx, np.float32)
    dx[1:] = gx[:-1] - gx[1:]
    gz0 = gz.copy()
    gz0[0] = 0.0
    ex = gz0[:, None, None] * dy[None, :, None] * gx[None, None, :]
    ey = gz0[:, None, None] * gy[None, :, None] * dx[None, None, :]
    return ex, ey


def pulse_run(name):
    """The full-size field runs: a configured workload's grid, materials and
    particle without the source and monitors, started from a curl_pulse
    centred on the particle, for a fixed number of steps.  Returns (prob,
    (E_x, E_y), steps)."""
    base, steps, width = {"cube_tips_au_gnor_512_pulse": ("cube_tips_au_gnor_512", 200, 24.0)}[name]
    prob = CONFIGS[base]()
    prob["source"] = None
    prob["monitors"] = None
    prob["steps"] = steps
    nx, ny, nz = prob["shape"]
    return prob, curl_pulse((nz, ny, nx), (nx / 2, ny / 2, nz / 2), (width,) * 3), steps


def small_sphere(n=36, radius_cells=5.0, pml=6, material=None, steps=200, band_ev=(1.0, 9.0), nf=16,
                 K=4, center_offset_half=(1, 0, -1), dx=0.5e-9, t0_tau=2.5):
    """A small test problem that spans several tiles and has ragged edges; the
    pulse is broad-band and starts early (t0 = t0_tau * tau) so short runs see it."""
    mat = material if material is not None else AU_LIKE_GNOR
    prob = sphere_problem(n, dx, radius_cells * dx, pml, mat, steps, band_ev, nf, K,
                          center_offset_half=center_offset_half)
    prob["source"]["t0"] = t0_tau * prob["source"]["tau"]
    return prob


# ------------------------------------------------------- batched / serving

def _dimer_or_sphere(rng, dx, kind):
    r = rng.uniform(1e-9, 6e-9)
    if kind == "sphere":
        R = half_cells(r, dx)
        ext = 2 * R
        return ext, [(0, R)]
    gap = rng.uniform(0.5e-9, 3e-9)
    R = half_cells(r, dx)
    G = half_cells(gap, dx)
    off = R + (G + 1) // 2                 # centre offset along x, half cells
    ext = 2 * (off + R)
    return ext, [(-off, R), (off, R)]


def batched_instances(n=64, seed=2005, dx=0.25e-9, steps=4000, pml=8, nf=200, K=16):
    """64 independent sphere/dimer solves on uneven grids 40^3..128^3."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        kind = "sphere" if rng.uniform() < 0.5 else "dimer"
        ext_half, spheres = _dimer_or_sphere(rng, dx, kind)
        beta = rng.uniform(0.9e6, 1.3e6)
        diff = 0.0 if rng.uniform() < 0.5 else rng.uniform(1e-4, 4e-4)
        side = max(40, int(math.ceil(ext_half / 2)) + 2 * (pml + PML_MARGIN_TF + METAL_MARGIN) + 2)
        if side > 128:
            continue
        mat = drude_material(9.0, 0.02, beta=beta, diff=diff)
        c = side                                    # grid centre in half cells
        shapes = [sphere_shape((c + dxo, c, c), R) for dxo, R in spheres]
        reach_x = max(abs(dxo) + R for dxo, R in spheres)
        reach = max(R for _, R in spheres)
        prob = scatter_problem((side,) * 3, dx, pml, [mat], shapes, ((c, c, c), (reach_x, reach, reach)),
                               steps, (2.0, 6.0), nf, K)
        prob["name"] = "%s_%02d" % (kind, len(out))
        out.append(prob)
    return out


def serving_requests(n=256, seed=6997, rate=20.0, dx=0.25e-9, nf=200, K=16):
    """A finite Poisson stream of sphere / dimer / cube-with-tips solves."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while len(out) < n:
        t += rng.exponential(1.0 / rate)
        u = rng.uniform()
        kind = "sphere" if u < 0.4 else ("dimer" if u < 0.8 else "cube_tips")
        steps = int(rng.integers(2000, 8001))
        gnor = rng.uniform() < 0.5
        mat = drude_material(9.0, 0.07 if gnor else 0.02, beta=1.2e6, diff=1.9e-4 if gnor else 0.0)
        pml = 8
        if kind == "cube_tips":
            side_m = rng.uniform(4e-9, 40e-9)
            sh = cube_tips_shape((0, 0, 0), side_m, 0.2 * side_m, 0.15 * side_m, 0.05 * side_m + 0.5e-9, dx)
            reach = sh["side"] // 2 + sh["tip_height"]
            nside = int(math.ceil(reach)) + 2 * (pml + PML_MARGIN_TF + METAL_MARGIN) + 2
        else:
            ext_half, spheres = _dimer_or_sphere(rng, dx, kind)
            nside = int(math.ceil(ext_half / 2)) + 2 * (pml + PML_MARGIN_TF + METAL_MARGIN) + 2
        nside = min(320, max(48, nside))
        c = nside
        if kind == "cube_tips":
            sh["c"] = (c, c, c)
            shapes, ext = [sh], ((c, c, c), (reach,) * 3)
        else:
            shapes = [sphere_shape((c + dxo, c, c), R) for dxo, R in spheres]
            reach_x = max(abs(dxo) + R for dxo, R in spheres)
            reach = max(R for _, R in spheres)
            ext = ((c, c, c), (reach_x, reach, reach))
        try:
            prob = scatter_problem((nside,) * 3, dx, pml, [mat], shapes, ext, steps, (2.0, 6.0), nf, K)
        except ValueError:
            continue
        prob["name"] = "req_%03d_%s" % (len(out), kind)
        prob["arrival_s"] = t
        out.append(prob)
    return out


def cells(prob) -> int:
    nx, ny, nz = prob["shape"]
    return nx * ny * nz
