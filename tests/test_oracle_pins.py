"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests retypes an oracle formula.  The dispersion tests derive
characteristic polynomials by z-transforming the *discretised differential
equations* as the paper first writes them (central differences, the weighted
E average, BDF2 for the GNOR term), while the oracle runs the *solved* update
forms with the coefficient sets D_1..D_d, D_G1, D_G2, C_1p..C_p.  Each
polynomial is itself checked against the continuous model (Eqs. NonlocDrude,
GNOR, CritPoint) in the limit dt, dx -> 0.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import Polynomial as Poly

import oracle
from paper_2005_06997_gb300 import workloads as W

EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6
C0 = 1.0 / math.sqrt(EPS0 * MU0)
E_OFF = ((1, 0, 0), (0, 1, 0), (0, 0, 1))
H_OFF = ((0, 1, 1), (1, 0, 1), (1, 1, 0))
z = Poly([0.0, 1.0])


def periodic_problem(n3, dx, courant=0.5, materials=(), eps_b=1.0):
    return {"shape": tuple(n3), "dx": dx, "courant": courant, "pml": 0, "bc": ("periodic",) * 3,
            "eps_b": eps_b, "materials": list(materials), "shapes": [], "source": None, "monitors": None}


def positions(off, n3):
    nx, ny, nz = n3
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i + off[0] / 2.0, j + off[1] / 2.0, k + off[2] / 2.0


def all_metal(n3, mat_id=1):
    nx, ny, nz = n3
    return np.full((3, nz, ny, nx), mat_id, dtype=np.uint8)


def recurrence_residual(x, poly, start=0):
    c = np.asarray(poly.coef, dtype=np.float64)
    c = c / np.max(np.abs(c))
    d = len(c) - 1
    x = np.asarray(x)
    res = np.array([np.dot(c, x[m:m + d + 1]) for m in range(start, len(x) - d)])
    return np.max(np.abs(res)) / (np.max(np.abs(x)) * np.sum(np.abs(c)))


def roots_to_omega(poly, dt):
    return 1j * np.log(poly.roots().astype(complex)) / dt


u = Poly([1.0, 1.0])      # z = 1 + u: keeps roots near z = 1 well conditioned


def roots_u_to_omega(poly, dt):
    """Roots of a polynomial in u = z - 1, mapped to w with z = exp(-i w dt)."""
    return 1j * np.log1p(poly.roots().astype(complex)) / dt


# --------------------------------------------------------------- Yee / CFL

@pytest.mark.parametrize("eps_b,S", [(1.0, 0.5), (1.77, 0.45)])
def test_vacuum_oblique_plane_wave_matches_discrete_dispersion(eps_b, S):
    """Exact discrete plane wave in a background of relative permittivity
    eps_b: sin^2(w dt/2) = (S^2 / eps_b) sum_a sin^2(k_a dx/2),
    H = K x E / (mu0 Omega) with the discrete wave vector K and frequency Omega
    (Faraday's law; Ampere's with eps0 eps_b then fixes the dispersion)."""
    n3, dx = (16, 12, 10), 1e-8
    m = np.array([1, 2, 1])
    k = 2 * np.pi * m / (np.array(n3) * dx)
    s = np.sin(k * dx / 2)
    Kt = 2 / dx * s
    e = np.array([Kt[1], -Kt[0], 0.0])
    e /= np.linalg.norm(e)
    dt = S * dx / C0
    w = 2 / dt * math.asin(S * math.sqrt(np.sum(s ** 2) / eps_b))
    Om = 2 / dt * math.sin(w * dt / 2)
    h = np.cross(Kt, e) / (MU0 * Om)
    sim = oracle.Sim(periodic_problem(n3, dx, S, eps_b=eps_b))
    for c in range(3):
        x, y, zz = positions(E_OFF[c], n3)
        sim.array("E" + "xyz"[c])[:] = e[c] * np.cos(k[0] * x * dx + k[1] * y * dx + k[2] * zz * dx)
        x, y, zz = positions(H_OFF[c], n3)
        sim.array("H" + "xyz"[c])[:] = h[c] * np.cos(k[0] * x * dx + k[1] * y * dx + k[2] * zz * dx + w * dt / 2)
    N = 120
    sim.step(N)
    for c in range(3):
        x, y, zz = positions(E_OFF[c], n3)
        ph = k[0] * x * dx + k[1] * y * dx + k[2] * zz * dx
        errE = np.max(np.abs(sim.array("E" + "xyz"[c]) - e[c] * np.cos(ph - w * N * dt)))
        x, y, zz = positions(H_OFF[c], n3)
        ph = k[0] * x * dx + k[1] * y * dx + k[2] * zz * dx
        errH = np.max(np.abs(sim.array("H" + "xyz"[c]) - h[c] * np.cos(ph - w * (N - 0.5) * dt)))
        assert errE <= 1e-10 * np.max(np.abs(e)), (c, errE)
        assert errH <= 1e-10 * np.max(np.abs(h)), (c, errH)


@pytest.mark.parametrize("S,stable", [(0.577, True), (0.578, False)])
def test_cfl_bound(S, stable):
    """The 3D Yee leapfrog is stable iff S <= 1/sqrt(3) (= 0.57735)."""
    n3 = (8, 8, 8)
    sim = oracle.Sim(periodic_problem(n3, 1e-8, S))
    rng = np.random.default_rng(1)
    for c in range(3):
        sim.array("E" + "xyz"[c])[:] = rng.uniform(-1, 1, size=(8, 8, 8))
    e0 = sum(np.sum(sim.array("E" + "xyz"[c]) ** 2) for c in range(3))
    sim.step(400)
    e1 = sum(np.sum(sim.array("E" + "xyz"[c]) ** 2) for c in range(3))
    if stable:
        assert e1 < 10 * e0
    else:
        assert e1 > 1e10 * e0


@pytest.mark.parametrize("b,stable", [(0.999, True), (1.001, False)])
def test_hydrodynamic_stability_bound(b, stable):
    """The pressure term of Eq. NonlocalUpdate adds beta^2 dt^2 K^2 / 4 to
    sin^2(w dt / 2) of a longitudinal mode (the discrete relation of the
    longitudinal-plasmon pin); with K^2 at most 12 / dx^2 (the (1,1,1)
    Nyquist mode of an even periodic grid, which has no curl and so no H)
    the scheme is stable iff beta dt sqrt(3) / dx <= 1, whatever wp (the
    (1,2,1)/4 average keeps the wp term stable).  Metal-filled periodic box,
    random E, beta set to b dx / (sqrt(3) dt)."""
    n3, dx = (8, 8, 8), 1e-9
    probe = oracle.Sim(periodic_problem(n3, dx, 0.5))
    beta = b * dx / (math.sqrt(3) * probe.dt)
    mat = {"eps_inf": 1.0, "wp": W.ev(9.0), "gamma": 0.0, "beta": beta, "diff": 0.0}
    sim = oracle.Sim(periodic_problem(n3, dx, 0.5, [mat]), all_metal(n3))
    rng = np.random.default_rng(3)
    for c in "xyz":
        sim.array("E" + c)[:] = rng.uniform(-1, 1, size=(8, 8, 8))
    e0 = sum(np.sum(sim.array("E" + c) ** 2) for c in "xyz")
    sim.step(400)
    e1 = sum(np.sum(sim.array("E" + c) ** 2) for c in "xyz")
    if stable:
        assert e1 < 10 * e0
    else:
        assert e1 > 1e10 * e0


# ------------------------------------------------- free-electron responses

def drude_lhs(dt, gamma, v=z):
    """z * [central-difference d2/dt2 + gamma central d/dt] of the P equation,
    as a polynomial in z (v = z) or in u = z - 1 (v = u)."""
    return (v - 1) ** 2 / dt ** 2 + gamma * (v ** 2 - 1) / (2 * dt)


def test_local_drude_transverse_wave_recurrence():
    """Transverse wave along z in homogeneous Drude metal (beta has no effect on
    a divergence-free P).  Eliminating H and P from the z-transformed Faraday,
    Ampere (Eq. discreteamperes) and the centred Drude equation with the
    (E^{n-1}+2E^n+E^{n+1})/4 average gives a quartic in z."""
    n3, dx, S = (2, 2, 32), 0.5e-9, 0.5
    wp, g, eps_inf = W.ev(9.0), W.ev(0.3), 1.5
    mat = {"eps_inf": eps_inf, "wp": wp, "gamma": g, "beta": 1.2e6, "diff": 0.0}
    sim = oracle.Sim(periodic_problem(n3, dx, S, [mat]), all_metal(n3))
    kz = 2 * np.pi / (n3[2] * dx)
    x, y, zz = positions(E_OFF[0], n3)
    sim.array("Ex")[:] = np.cos(kz * zz * dx)
    dt = sim.dt
    series = []
    for _ in range(300):
        series.append(sim.array("Ex")[5, 0, 0])
        sim.step(1)
    s2 = math.sin(kz * dx / 2) ** 2
    A = drude_lhs(dt, g)
    B = EPS0 * wp ** 2 * (z + 1) ** 2 / 4
    char = (z - 1) ** 2 * (EPS0 * eps_inf * A + B) + (4 * s2 * dt ** 2 / (MU0 * dx ** 2)) * z * A
    assert recurrence_residual(series, char, start=1) < 1e-11
    # the polynomial itself tends to k^2 c^2 = w^2 eps(w) of the local Drude model
    lam = 300e-9
    kk = 2 * np.pi / lam
    dxf = lam / 20000
    dtf = 0.5 * dxf / C0
    s2f = math.sin(kk * dxf / 2) ** 2
    A = drude_lhs(dtf, g, u)
    B = EPS0 * wp ** 2 * (u + 1) ** 2 / 4
    charf = (u - 1) ** 2 * (EPS0 * eps_inf * A + B) + (4 * s2f * dtf ** 2 / (MU0 * dxf ** 2)) * u * A
    wd = roots_u_to_omega(charf, dtf)
    # continuum: eps_inf w^3 + i g eps_inf w^2 - (wp^2 + k^2 c^2) w - i g k^2 c^2 = 0
    wc = np.roots([eps_inf, 1j * g * eps_inf, -(wp ** 2 + kk ** 2 * C0 ** 2), -1j * g * kk ** 2 * C0 ** 2])
    for r in wc:
        if abs(r) < 1e-3 * wp:
            continue
        assert np.min(np.abs(wd - r)) / abs(r) < 1e-4


def longitudinal_setup(n3, dx, m, mat, S=0.5):
    """Metal everywhere, P along the discrete wave vector, E = -P/(eps0 eps_inf), H = 0."""
    sim = oracle.Sim(periodic_problem(n3, dx, S, [mat]), all_metal(n3))
    k = 2 * np.pi * np.asarray(m) / (np.asarray(n3) * dx)
    s = np.sin(k * dx / 2)
    pol = s / np.linalg.norm(s)
    for c in range(3):
        x, y, zz = positions(E_OFF[c], n3)
        P = 1e-11 * pol[c] * np.cos(k[0] * x * dx + k[1] * y * dx + k[2] * zz * dx)
        sim.array("P" + "xyz"[c])[:] = P
        sim.array("E" + "xyz"[c])[:] = -P / (EPS0 * mat["eps_inf"])
    K2 = np.sum((2 / dx * s) ** 2)
    return sim, K2, pol


@pytest.mark.parametrize("m", [(2, 0, 0), (1, 2, 0)], ids=["axis", "oblique"])
def test_nonlocal_longitudinal_plasmon(m):
    """Eq. NonlocDrude for a longitudinal mode: grad(div P) = -K^2 P (discrete K),
    E = -P/(eps0 eps_inf).  The oblique case exercises the mixed differences of
    Eq. GradDiv.  Closed form at gamma = 0: sin^2(w dt/2) = (a+b)/(1+a) with
    a = dt^2 wp^2/(4 eps_inf), b = dt^2 beta^2 K^2/4; continuum w^2 = wp^2/eps_inf + beta^2 k^2."""
    n3 = (32, 2, 2) if m[1] == 0 else (16, 16, 2)
    dx = 0.1e-9
    wp, beta, eps_inf = W.ev(9.0), 1.07e6, 1.3
    for g in (0.0, W.ev(0.2)):
        mat = {"eps_inf": eps_inf, "wp": wp, "gamma": g, "beta": beta, "diff": 0.0}
        sim, K2, pol = longitudinal_setup(n3, dx, m, mat)
        dt = sim.dt
        comp = 0
        series = []
        for _ in range(240):
            series.append(sim.array("Px")[1, 1, 3])
            sim.step(1)
        char = drude_lhs(dt, g) + wp ** 2 * (z + 1) ** 2 / (4 * eps_inf) + beta ** 2 * K2 * z
        assert recurrence_residual(series, char) < 1e-11
        eta0 = math.sqrt(MU0 / EPS0)
        hmax = max(np.max(np.abs(sim.array(n))) for n in ("Hx", "Hy", "Hz"))
        assert hmax < 1e-9 * np.max(np.abs(sim.array("Ex"))) / eta0
        if g == 0.0:
            a = dt ** 2 * wp ** 2 / (4 * eps_inf)
            b = dt ** 2 * beta ** 2 * K2 / 4
            w = roots_to_omega(char, dt)
            w = np.max(np.abs(w.real))
            assert abs(math.sin(w * dt / 2) ** 2 - (a + b) / (1 + a)) < 1e-12
    # continuum limit of the same polynomial
    kk = 2 * np.pi / 2e-9
    dtf = 1e-21
    char = drude_lhs(dtf, 0.0, u) + wp ** 2 * (u + 1) ** 2 / (4 * eps_inf) + beta ** 2 * kk ** 2 * u
    w = np.max(np.abs(roots_u_to_omega(char, dtf).real))
    assert abs(w ** 2 / (wp ** 2 / eps_inf + beta ** 2 * kk ** 2) - 1) < 1e-6


@pytest.mark.parametrize("m", [(2, 0, 0), (1, 2, 0)], ids=["axis", "oblique"])
def test_gnor_longitudinal_plasmon(m):
    """Eq. GNOR with the BDF2 time derivative of grad(div P): the z-transform is a
    cubic.  Its roots tend to w^2 + i g w = wp^2/eps_inf + (beta^2 + D g - i D w) k^2,
    the substitution the paper uses for diffusive Mie theory."""
    n3 = (32, 2, 2) if m[1] == 0 else (16, 16, 2)
    dx = 0.1e-9
    wp, g, beta, D, eps_inf = W.ev(9.0), W.ev(0.1), 1.2e6, 3.61e-4, 1.0
    mat = {"eps_inf": eps_inf, "wp": wp, "gamma": g, "beta": beta, "diff": D}
    sim, K2, pol = longitudinal_setup(n3, dx, m, mat)
    dt = sim.dt
    series = []
    for _ in range(240):
        series.append(sim.array("Px")[1, 1, 3])
        sim.step(1)
    eta = beta ** 2 + D * g

    def gnor_char(dt, K2, v=z):
        lhs = ((v - 1) ** 2 / dt ** 2 + g * (v ** 2 - 1) / (2 * dt)) * v
        rhs_e = -wp ** 2 * (v + 1) ** 2 * v / (4 * eps_inf)       # eps0 wp^2 <E> with E = -P/(eps0 eps_inf)
        rhs_gd = -K2 * (eta * v ** 2 + D * (3 * v ** 2 - 4 * v + 1) / (2 * dt))
        return lhs - rhs_e - rhs_gd

    assert recurrence_residual(series, gnor_char(dt, K2)) < 1e-11
    kk = 2 * np.pi / 2e-9
    dtf = 1e-21
    wd = roots_u_to_omega(gnor_char(dtf, kk ** 2, u), dtf)
    # continuum: w^2 + i(g + D k^2) w - (wp^2/eps_inf + (beta^2 + D g) k^2) = 0
    wc = np.roots([1.0, 1j * (g + D * kk ** 2), -(wp ** 2 / eps_inf + (beta ** 2 + D * g) * kk ** 2)])
    for r in wc:
        assert np.min(np.abs(wd - r)) / abs(r) < 1e-5


def cp_discrete_chi(zv, dt, A, Om, Ga, phi):
    """chi_d(z) = P/(eps0 E) of the critical-points ODE
    P'' + 2 Ga P' + (Om^2+Ga^2) P = 2 eps0 A Om [(Om cos phi - Ga sin phi) E - sin phi E'],
    centred at n with the (1,2,1)/4 average on P and E (Eq. CritPoint under exp(-iwt))."""
    lhs = (zv - 1) ** 2 / dt ** 2 + Ga * (zv ** 2 - 1) / dt + (Om ** 2 + Ga ** 2) * (zv + 1) ** 2 / 4
    rhs = 2 * A * Om * ((Om * np.cos(phi) - Ga * np.sin(phi)) * (zv + 1) ** 2 / 4 - np.sin(phi) * (zv ** 2 - 1) / (2 * dt))
    return rhs / lhs


def chi_cp(w, A, Om, Ga, phi):
    return A * Om * (np.exp(1j * phi) / (Om - w - 1j * Ga) + np.exp(-1j * phi) / (Om + w + 1j * Ga))


@pytest.mark.parametrize("phi", [0.0, 0.35])
def test_critical_point_pole(phi):
    """Eq. critpointupdate: a homogeneous k = 0 oscillation (curl H = 0 so
    eps0 eps_inf E + P_CP = 0) obeys the quadratic of the discretised CP
    equation; that discretisation tends to chi_CP of Eq. CritPoint, and the
    update's fixed point is exactly eps0 chi_CP(0) E."""
    n3, dx = (2, 2, 2), 0.2e-9
    A, Om, Ga, eps_inf = 1.5, W.ev(4.0), W.ev(0.5), 2.0
    mat = {"eps_inf": eps_inf, "wp": 0.0, "gamma": 0.0, "beta": 0.0, "diff": 0.0,
           "poles": [(A, Om, Ga, phi)]}
    sim = oracle.Sim(periodic_problem(n3, dx, 0.5, [mat]), all_metal(n3))
    sim.array("Pcpx")[:] = 1e-11
    sim.array("Ex")[:] = -1e-11 / (EPS0 * eps_inf)
    dt = sim.dt
    series = []
    for _ in range(200):
        series.append(sim.array("Pcpx")[0, 0, 0])
        sim.step(1)
    lhs = (z - 1) ** 2 / dt ** 2 + Ga * (z ** 2 - 1) / dt + (Om ** 2 + Ga ** 2) * (z + 1) ** 2 / 4
    rhs = 2 * A * Om * ((Om * math.cos(phi) - Ga * math.sin(phi)) * (z + 1) ** 2 / 4
                        - math.sin(phi) * (z ** 2 - 1) / (2 * dt))
    char = lhs + rhs / eps_inf
    assert recurrence_residual(series, char) < 1e-11
    for wv in (W.ev(1.0), W.ev(3.5), W.ev(6.0)):
        dtf = 1e-21
        zv = np.exp(-1j * wv * dtf)
        assert abs(cp_discrete_chi(zv, dtf, A, Om, Ga, phi) / chi_cp(wv, A, Om, Ga, phi) - 1) < 1e-5
    c = sim.coefficients(1)["poles"][0]
    chi0 = (c["C3"] + c["C4"] + c["C5"]) / (1 - c["C1"] - c["C2"]) / EPS0
    # 1 - C1 - C2 cancels to (Om^2+Ga^2)/Cp ~ (Om dt)^2: FP64 leaves ~1e-11 relative
    assert abs(chi0 - chi_cp(0.0, A, Om, Ga, phi).real) < 1e-9 * abs(chi0)


def test_drude_coefficients_sum_to_one():
    """D1 + D2 = 1 (Eqs. d1, d2, dd), which the increment form of the update relies on."""
    mat = {"eps_inf": 1.0, "wp": W.ev(9.0), "gamma": W.ev(0.07), "beta": 1.2e6, "diff": 1.9e-4}
    sim = oracle.Sim(periodic_problem((2, 2, 2), 0.2e-9, 0.5, [mat]), all_metal((2, 2, 2)))
    d = sim.coefficients(1)
    assert abs(d["D1"] + d["D2"] - 1.0) < 1e-15


# ------------------------------------------------------- operator identities

def test_graddiv_is_symmetric_and_negative():
    """Summation by parts: <Q, GD(P)> = <GD(Q), P> and <P, GD(P)> = -sum_nodes (div P)^2
    for P, Q vanishing off the metal (Pekar), with div the plain node divergence."""
    n3 = (14, 13, 12)
    dx = 0.3e-9
    prob = {"shape": n3, "dx": dx, "courant": 0.5, "pml": 0, "bc": ("pec",) * 3, "eps_b": 1.0,
            "materials": [W.AG_LIKE], "shapes": [W.sphere_shape((14, 13, 12), 8)],
            "source": None, "monitors": None}
    sim = oracle.Sim(prob)
    mask = sim.material_map() > 0
    rng = np.random.default_rng(7)
    P = [rng.standard_normal(mask[c].shape) * mask[c] for c in range(3)]
    Q = [rng.standard_normal(mask[c].shape) * mask[c] for c in range(3)]
    GP = sim.graddiv(P)
    GQ = sim.graddiv(Q)
    lhs = sum(np.sum(Q[c] * GP[c]) for c in range(3))
    rhs = sum(np.sum(GQ[c] * P[c]) for c in range(3))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # node divergence d(i,j,k) = sum_a P_a(node) - P_a(node - e_a), zero outside the grid
    nx, ny, nz = n3
    d = np.zeros((nz + 1, ny + 1, nx + 1))
    for c, sl in enumerate([(slice(None), slice(None), slice(0, nx)), (slice(None), slice(0, ny), slice(None)),
                            (slice(0, nz), slice(None), slice(None))]):
        Pp = np.zeros((nz + 1, ny + 1, nx + 1))
        Pp[:nz, :ny, :nx] = P[c]
        sh = [0, 0, 0]
        sh[2 - c] = 1
        Pm = np.roll(Pp, shift=sh, axis=(0, 1, 2))
        d += Pp - Pm
    energy = sum(np.sum(P[c] * GP[c]) for c in range(3))
    assert energy < 0
    assert abs(energy + np.sum(d ** 2) / dx ** 2) < 1e-12 * abs(energy)


def test_ampere_law_holds_and_pekar():
    """After every step eps0 eps_inf dE + dP_f + dP_CP = dt curl H^{n+1/2} at each
    interior E-site (Eq. discreteamperes; this fixes the sign of C4p, reading 1),
    and P_f stays exactly zero off the metal (Pekar ABC)."""
    prob = W.small_sphere(n=36, steps=0)
    sim = oracle.Sim(prob)
    sim.step(60)
    mp = sim.material_map()
    dx, dt = prob["dx"], sim.dt
    mat = prob["materials"][0]
    for _ in range(3):
        sim.step(1)
        Hx, Hy, Hz = (sim.array(n) for n in ("Hx", "Hy", "Hz"))
        curl = [
            (Hz - np.roll(Hz, 1, axis=1)) - (Hy - np.roll(Hy, 1, axis=0)),
            (Hx - np.roll(Hx, 1, axis=0)) - (Hz - np.roll(Hz, 1, axis=2)),
            (Hy - np.roll(Hy, 1, axis=2)) - (Hx - np.roll(Hx, 1, axis=1)),
        ]
        for c in range(3):
            a = "xyz"[c]
            metal = mp[c] > 0
            eps = np.where(metal, mat["eps_inf"], 1.0)
            lhs = (EPS0 * eps * (sim.array("E" + a) - sim.array("E" + a + "_prev"))
                   + (sim.array("P" + a) - sim.array("P" + a + "_prev"))
                   + (sim.array("Pcp" + a) - sim.array("Pcp" + a + "_prev")))
            rhs = dt * curl[c] / dx
            sl = (slice(13, 23),) * 3          # inside the TF box, away from the CPML
            err = np.max(np.abs(lhs[sl] - rhs[sl]))
            scale = np.max(np.abs(dt * np.abs(curl[c][sl]) / dx)) + np.max(np.abs(EPS0 * sim.array("E" + a)[sl]))
            assert metal[sl].any()
            assert err <= 1e-12 * scale, (c, err, scale)
            assert np.all(sim.array("P" + a)[~metal] == 0.0)


# ------------------------------------------------------------ TF/SF, CPML

@pytest.mark.parametrize("eps_b,S", [(1.0, 0.5), (1.77, 0.45)])
def test_tfsf_no_leakage_without_scatterer(eps_b, S):
    """Axis-aligned incidence with a matched 1D grid (same background, same
    Courant number): the scattered-field region stays empty up to rounding."""
    prob = W.small_sphere(n=36, steps=0)
    prob["shapes"] = []
    prob["eps_b"], prob["courant"] = eps_b, S
    prob["monitors"] = None
    prob["dx"] = 1e-9
    src = dict(prob["source"])
    src["t0"] = 2.5 * src["tau"]
    prob["source"] = src
    sim = oracle.Sim(prob)
    lo, hi = src["tf_lo"], src["tf_hi"]
    worst = 0.0
    peak = 0.0
    for _ in range(8):
        sim.step(100)
        Ex = sim.array("Ex")
        nz, ny, nx = Ex.shape
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        tf = (i >= lo[0]) & (i <= hi[0] - 1) & (j >= lo[1]) & (j <= hi[1]) & (k >= lo[2]) & (k <= hi[2])
        peak = max(peak, np.max(np.abs(Ex[tf])))
        sf = max(np.max(np.abs(Ex[~tf])), np.max(np.abs(sim.array("Ey"))), np.max(np.abs(sim.array("Ez"))))
        worst = max(worst, sf)
    assert peak > 1e-3
    assert worst <= 1e-13 * peak


def test_cpml_normal_incidence_reflection():
    """A plane-wave pulse into the CPML (reading 7, 10 cells): the reflected
    field is below -40 dB of the incident one (compared against a run whose
    far wall is out of reach)."""
    dx, S, L = 1e-9, 0.5, 10

    def run(nz):
        prob = {"shape": (2, 2, nz), "dx": dx, "courant": S, "pml": L, "bc": ("periodic", "periodic", "cpml"),
                "eps_b": 1.0, "materials": [], "shapes": [], "source": None, "monitors": None}
        sim = oracle.Sim(prob)
        dt = sim.dt
        k = np.arange(nz)
        z0, w = 40.0, 6.0
        sim.array("Ex")[:] = np.exp(-((k - z0) / w) ** 2)[:, None, None]
        # matching H for +z travel, half a step earlier and half a cell up
        zh = k + 0.5 + 0.5 * S
        sim.array("Hy")[:] = (np.exp(-((zh - z0) / w) ** 2) / math.sqrt(MU0 / EPS0))[:, None, None]
        sim.step(260)
        return sim.array("Ex")[:, 0, 0].copy()

    a = run(100)
    b = run(400)
    ref = np.max(np.abs(b[15:85]))
    refl = np.max(np.abs(a[15:85] - b[15:85]))
    assert ref > 0.0
    assert refl < 1e-2 * 1.0


# ---------------------------------------------------------------- geometry

def brute_inside(shape, p):
    """The shape definitions restated on exact rationals (cell units)."""
    c = [Fraction(v, 2) for v in shape["c"]]
    x = [Fraction(v, 2) for v in p]
    d = [x[a] - c[a] for a in range(3)]
    if shape["kind"] == "sphere":
        return sum(v * v for v in d) <= Fraction(shape["radius"], 2) ** 2
    if shape["kind"] == "cube_tips":
        A = Fraction(shape["side"], 4)
        B = Fraction(shape["tip_base"], 4)
        h = Fraction(shape["tip_height"], 2)
        if all(abs(v) <= A for v in d):
            return True
        for ax in range(3):
            for sgn in (-1, 1):
                t = sgn * d[ax]
                v, w = abs(d[(ax + 1) % 3]), abs(d[(ax + 2) % 3])
                tc = Fraction(shape["tip_center"], 2)
                if (t - tc) ** 2 + v * v + w * w <= Fraction(shape["tip_radius"], 2) ** 2:
                    return True
                # pyramid: half width B at the face t = A, shrinking linearly to 0 at t = A + h
                if A <= t <= Fraction(shape["tip_cut"], 2):
                    half = B * (A + h - t) / h
                    if v <= half and w <= half:
                        return True
        return False
    raise ValueError


@pytest.mark.parametrize("kind", ["sphere", "cube_tips"])
def test_voxeliser_brute_force(kind):
    n3 = (13, 12, 14)
    if kind == "sphere":
        shape = W.sphere_shape((13, 11, 15), 9)
    else:
        shape = {"kind": "cube_tips", "material": 1, "c": (13, 12, 14), "side": 8, "tip_base": 6,
                 "tip_height": 6, "tip_radius": 2, "tip_center": 8, "tip_cut": 9}
    prob = {"shape": n3, "dx": 1e-9, "courant": 0.5, "pml": 0, "bc": ("pec",) * 3, "eps_b": 1.0,
            "materials": [W.AG_LIKE], "shapes": [shape], "source": None, "monitors": None}
    mp = oracle.Sim(prob).material_map()
    nx, ny, nz = n3
    for c in range(3):
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    p = (2 * i + E_OFF[c][0], 2 * j + E_OFF[c][1], 2 * k + E_OFF[c][2])
                    assert (mp[c, k, j, i] == 1) == brute_inside(shape, p), (c, i, j, k)


def test_voxeliser_sphere_volume():
    R_cells = 10
    n3 = (26, 26, 26)
    prob = {"shape": n3, "dx": 1e-9, "courant": 0.5, "pml": 0, "bc": ("pec",) * 3, "eps_b": 1.0,
            "materials": [W.AG_LIKE], "shapes": [W.sphere_shape((26, 26, 26), 2 * R_cells)],
            "source": None, "monitors": None}
    mp = oracle.Sim(prob).material_map()
    vol = 4.0 / 3.0 * math.pi * R_cells ** 3
    for c in range(3):
        assert abs(np.count_nonzero(mp[c]) / vol - 1.0) < 0.02
    # the three components see the same sphere up to the cyclic relabelling
    assert np.count_nonzero(mp[0]) == np.count_nonzero(mp[1]) == np.count_nonzero(mp[2])


# ------------------------------------------------------------------- energy

def discrete_energy_series(mat, steps, n=10, dx=0.5e-9, seed=7):
    """Metal-filled PEC box, random initial E (tangential E zero on the walls),
    H = P = 0, no source.  Per step: the electromagnetic energy
    eps0 eps_inf |E^n|^2 / 2 + mu0 H^{n-1/2}.H^{n+1/2} / 2 (the quantity the Yee
    scheme conserves in vacuum) plus the free-electron kinetic energy
    |J^{n+1/2}|^2 / (2 eps0 wp^2) with J^{n+1/2} = (P^{n+1} - P^n)/dt and the
    pressure energy beta^2 (div P^n)(div P^{n+1}) / (2 eps0 wp^2), summed over
    the sites (the continuum energy of Eq. NonlocDrude; uniform cells, so the
    cell volume is left out)."""
    n3 = (n, n, n)
    prob = {"shape": n3, "dx": dx, "courant": 0.5, "pml": 0, "bc": ("pec",) * 3, "eps_b": 1.0,
            "materials": [mat], "shapes": [], "source": None, "monitors": None}
    sim = oracle.Sim(prob, all_metal(n3))
    rng = np.random.default_rng(seed)
    for c in "xyz":
        sim.array("E" + c)[:] = rng.standard_normal(sim.shape3)
    sim.array("Ex")[:, 0, :] = 0
    sim.array("Ex")[0, :, :] = 0
    sim.array("Ey")[:, :, 0] = 0
    sim.array("Ey")[0, :, :] = 0
    sim.array("Ez")[:, :, 0] = 0
    sim.array("Ez")[:, 0, :] = 0
    wp2, beta, dt, eps_inf = mat["wp"] ** 2, mat["beta"], sim.dt, mat["eps_inf"]
    H0 = [np.array(sim.array("H" + c)) for c in "xyz"]
    P0 = [np.array(sim.array("P" + c)) for c in "xyz"]
    d0 = sim.density()
    out = np.empty(steps)
    for s in range(steps):
        E = [np.array(sim.array("E" + c)) for c in "xyz"]
        sim.step(1)
        H1 = [np.array(sim.array("H" + c)) for c in "xyz"]
        P1 = [np.array(sim.array("P" + c)) for c in "xyz"]
        d1 = sim.density()
        w = 0.5 * EPS0 * eps_inf * sum(np.sum(e * e) for e in E)
        w += 0.5 * MU0 * sum(np.sum(a * b) for a, b in zip(H0, H1))
        w += 0.5 * sum(np.sum(((a - b) / dt) ** 2) for a, b in zip(P1, P0)) / (EPS0 * wp2)
        w += 0.5 * beta ** 2 * np.sum(d0 * d1) / (EPS0 * wp2)
        out[s] = w
        H0, P0, d0 = H1, P1, d1
    return out


@pytest.mark.parametrize("case", ["lossless", "lossy", "gnor"])
def test_energy_bounded_without_loss_and_decaying_with_it(case):
    """Without damping (gamma = D = 0) the energy of the coupled system stays
    where it started (averaged over windows of 500 steps, within 0.1 %; a
    growing mode, e.g. a coupling of the wrong sign, fails this); with gamma
    (and with the GNOR diffusion term) it decreases from window to window."""
    gamma, diff = {"lossless": (0.0, 0.0), "lossy": (0.3, 0.0), "gnor": (0.3, 1.9e-4)}[case]
    mat = W.drude_material(9.0, gamma, beta=1.07e6, diff=diff)
    w = discrete_energy_series(mat, 8000)
    win = w.reshape(-1, 500).mean(axis=1)
    if case == "lossless":
        assert np.max(np.abs(win / win[0] - 1)) < 1e-3
    else:
        assert np.all(np.diff(win) < 0)
        assert win[-1] < 0.9 * win[0]


# ------------------------------------------------ nonlocal metal in the CPML

def cpml_slab_problem(beta=3.6e6, diff=1.9e-4, n=(32, 16, 16), pml=8):
    """A GNOR slab (a substrate-like box) running along x through the CPML
    at both ends of a grid with a CPML on x and PEC walls on y and z; no
    source (the initial field is set by blob_init)."""
    mat = W.drude_material(9.0, 0.07, beta=beta, diff=diff)
    nx, ny, nz = n
    sh = {"kind": "box", "material": 1, "c": (nx, ny, nz), "half": (nx - 5, 4, 4)}
    return {"shape": n, "dx": 0.25e-9, "courant": 0.5, "pml": pml, "bc": ("cpml", "pec", "pec"), "eps_b": 1.0,
            "materials": [mat], "shapes": [sh], "source": None, "monitors": None, "steps": 0}


def blob_init(sim):
    """A smooth E_x, E_y blob around the grid centre (walls excluded)."""
    Ex, Ey = sim.array("Ex"), sim.array("Ey")
    nz, ny, nx = Ex.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    blob = np.exp(-(((i - nx / 2) / 4.0) ** 2 + ((j - ny / 2 - 0.5) / 3.0) ** 2 + ((k - nz / 2) / 3.0) ** 2))
    Ey[1:, :, 1:] = blob[1:, :, 1:]
    Ex[1:, 1:, :] = 0.5 * blob[1:, 1:, :]


def test_nonlocal_metal_in_the_cpml_is_local_drude_there():
    """Sec. III keeps the nonlocal response out of the PML: a nonlocal metal
    reaching into it is updated there with the local Drude model.  The oracle
    run of the GNOR slab must equal, bit for bit, the run of an explicit
    material map that gives every E-site of a CPML cell a second material,
    the same metal with beta = D = 0 (and the GNOR one elsewhere)."""
    prob = cpml_slab_problem()
    a = oracle.Sim(prob)
    vox = a.material_map()
    nz, ny, nx = vox.shape[1:]
    L = prob["pml"]
    in_pml = np.zeros((nz, ny, nx), dtype=bool)
    in_pml[:, :, :L] = True
    in_pml[:, :, nx - L:] = True
    assert np.any(vox[:, in_pml]) and np.any(vox[:, ~in_pml])
    local = dict(prob["materials"][0], beta=0.0, diff=0.0)
    twin = dict(prob, materials=[prob["materials"][0], local], shapes=[])
    mp = vox.copy()
    mp[:, in_pml] = np.where(vox[:, in_pml] > 0, 2, 0)
    b = oracle.Sim(twin, material_map=mp)
    blob_init(a)
    blob_init(b)
    a.step(600)
    b.step(600)
    for f in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "Px", "Py", "Pz"):
        assert np.array_equal(a.array(f), b.array(f)), f
    assert np.max(np.abs(a.array("Px"))) > 0


def test_slab_through_the_cpml_stays_bounded():
    """With the local model inside the CPML the slab's field energy stays
    bounded over 10^4 steps (the same run with the nonlocal terms kept in the
    CPML grows without bound: five-fold by step 8000 on this grid)."""
    prob = cpml_slab_problem()
    s = oracle.Sim(prob)
    blob_init(s)
    e2 = []
    for _ in range(20):
        s.step(500)
        e2.append(sum(float(np.sum(np.asarray(s.array(c)) ** 2)) for c in ("Ex", "Ey", "Ez")))
    assert max(e2[-4:]) <= 1.5 * max(e2[:4]), e2
