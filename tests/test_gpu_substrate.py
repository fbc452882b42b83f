"""A nonlocal structure that extends through the PML (Sec. III: it follows
the local Drude model inside the PML), on the GPU against the FP64 oracle.

A GNOR slab runs along x through the CPML at both ends of a grid with a
CPML on x and PEC walls on y and z, like a substrate; a smooth initial field
(no source) excites it.  The GPU's CPML material sites take the CPML's psi
terms in their curl and drop the pressure and diffusion terms."""
import numpy as np
import pytest

import oracle
from paper_2005_06997_gb300 import nlfdtd
from paper_2005_06997_gb300 import workloads as W

pytestmark = pytest.mark.gpu

VECTORS = {"E": ("Ex", "Ey", "Ez"), "H": ("Hx", "Hy", "Hz"), "P": ("Px", "Py", "Pz")}


def slab_problem(beta=3.6e6, diff=1.9e-4, n=(32, 16, 16), pml=8):
    mat = W.drude_material(9.0, 0.07, beta=beta, diff=diff, poles=[W.lorentz_pole()])
    nx, ny, nz = n
    sh = {"kind": "box", "material": 1, "c": (nx, ny, nz), "half": (nx - 5, 4, 4)}
    return {"shape": n, "dx": 0.25e-9, "courant": 0.5, "pml": pml, "bc": ("cpml", "pec", "pec"), "eps_b": 1.0,
            "materials": [mat], "shapes": [sh], "source": None, "monitors": None, "steps": 0}


def blob(shape3):
    nz, ny, nx = shape3
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    b = np.exp(-(((i - nx / 2) / 4.0) ** 2 + ((j - ny / 2 - 0.5) / 3.0) ** 2 + ((k - nz / 2) / 3.0) ** 2))
    ey = np.zeros(shape3)
    ex = np.zeros(shape3)
    ey[1:, :, 1:] = b[1:, :, 1:]
    ex[1:, 1:, :] = 0.5 * b[1:, 1:, :]
    return ex, ey


def curl_blob(shape3):
    """A divergence-free initial E (the discrete curl of a Gaussian A z-hat,
    A at the cell's (i+1/2, j+1/2, k)): E_x = A(j) - A(j-1), E_y = A(i-1) -
    A(i), so that div E = 0 at every node and the pulse radiates (H reaches
    about E / eta0 instead of staying a small residual); tangential E zero
    on the walls."""
    nz, ny, nx = shape3
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a = np.exp(-(((i + 0.5 - nx / 2) / 4.0) ** 2 + ((j + 0.5 - ny / 2) / 3.0) ** 2 + ((k - nz / 2) / 3.0) ** 2))
    ex = np.zeros(shape3)
    ey = np.zeros(shape3)
    ex[:, 1:, :] = a[:, 1:, :] - a[:, :-1, :]
    ey[:, :, 1:] = a[:, :, :-1] - a[:, :, 1:]
    ex[0], ey[0] = 0.0, 0.0          # tangential E on the z = 0 wall
    ex[:, 0, :] = 0.0                # E_x on the y = 0 wall
    ey[:, :, 0] = 0.0                # E_y on the x = 0 wall
    return ex, ey


def start_pair(prob, init=blob):
    g = nlfdtd.Solver(prob)
    o = oracle.Sim(prob)
    ex, ey = init(o.shape3)
    o.array("Ex")[...] = ex
    o.array("Ey")[...] = ey
    g.set_field("Ex", ex)
    g.set_field("Ey", ey)
    return g, o


def test_slab_through_the_cpml_matches_oracle():
    prob = slab_problem()
    g, o = start_pair(prob)
    assert np.array_equal(g.field("Ey"), np.asarray(o.array("Ey"), dtype=np.float32))
    g.run(600)
    g.sync()
    o.step(600)
    for vec, comps in VECTORS.items():
        num = sum(np.sum((g.field(c).astype(np.float64) - o.array(c)) ** 2) for c in comps)
        den = sum(np.sum(np.asarray(o.array(c)) ** 2) for c in comps)
        assert den > 0, vec
        assert np.sqrt(num / den) <= 1e-4, (vec, np.sqrt(num / den))
    # the slab's P_f is alive inside the CPML cells too
    px = np.asarray(o.array("Px"))
    assert np.max(np.abs(px[:, :, :8])) > 1e-3 * np.max(np.abs(px))
    g.close()


def test_slab_through_the_cpml_stays_bounded_on_the_gpu():
    prob = slab_problem()
    g, _ = start_pair(prob)
    e2 = []
    for _ in range(20):
        g.run(500)
        g.sync()
        e2.append(sum(float(np.sum(g.field(c).astype(np.float64) ** 2)) for c in ("Ex", "Ey", "Ez")))
    assert max(e2[-4:]) <= 1.5 * max(e2[:4]), e2
    g.close()


@pytest.mark.parametrize("n3,bc,half", [
    ((36, 20, 47), ("cpml", "cpml", "cpml"), (24, 14, 42)),
    ((40, 16, 16), ("pec", "pec", "cpml"), (32, 8, 11)),
], ids=["ragged_interior", "thinnest_grid"])
def test_z_chunks_with_metal_through_the_z_cpml(n3, bc, half):
    """The z chunks of the EM march with a CPML along z: the end chunks hold
    the slab and one plane more, the interior ones kz planes (47 planes with
    a 6-cell CPML: seven, then 8 + 8 + 8 + 8 + 1, then seven); the thinnest
    grid a 6-cell CPML allows (16 planes) leaves a two-plane interior chunk.
    A one-pole GNOR block that fills at least a quarter of the grid (so its
    tiles update their sites inside the z march) runs through the z CPML
    (local Drude there, sites of CPML tiles on the site list)."""
    mat = W.drude_material(9.0, 0.07, beta=3.6e6, diff=1.9e-4, poles=[W.lorentz_pole()])
    nx, ny, nz = n3
    sh = {"kind": "box", "material": 1, "c": (nx, ny, nz), "half": half}
    prob = {"shape": n3, "dx": 0.25e-9, "courant": 0.5, "pml": 6, "bc": bc, "eps_b": 1.0,
            "materials": [mat], "shapes": [sh], "source": None, "monitors": None, "steps": 0}
    g, o = start_pair(prob, curl_blob)
    g.run(300)
    g.sync()
    o.step(300)
    # E and P_f as vector fields; H in the field's own norm (eta0 H against
    # E and eta0 H together): what remains after 300 steps is mostly the
    # block's near field, where H is a small part of the field and its own
    # relative error is the FP32 rounding of E's curl
    eta0 = 376.730313668
    sq = lambda f, c: np.sum(np.asarray(f(c), dtype=np.float64) ** 2)
    d2 = {v: sum(np.sum((g.field(c).astype(np.float64) - o.array(c)) ** 2) for c in comps)
          for v, comps in VECTORS.items()}
    r2 = {v: sum(sq(o.array, c) for c in comps) for v, comps in VECTORS.items()}
    assert all(r2[v] > 0 for v in VECTORS), r2
    errs = {"E": np.sqrt(d2["E"] / r2["E"]), "P": np.sqrt(d2["P"] / r2["P"]),
            "H": eta0 * np.sqrt(d2["H"] / (r2["E"] + eta0 ** 2 * r2["H"]))}
    assert all(e <= 1e-4 for e in errs.values()), errs
    pz = np.asarray(o.array("Pz"))
    assert np.max(np.abs(pz[:6])) > 1e-4 * np.max(np.abs(pz))       # the block is alive in the z CPML
    g.close()
