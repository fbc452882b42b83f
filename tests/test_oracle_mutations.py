"""Planted mistakes: each one, applied to a copy of oracle/oracle.c, must make
at least one of the pins fail.  The oracle's own source is never modified;
every mutant is built into a temporary directory and loaded by a pytest
subprocess through the ORACLE_LIB override, which runs only the pins named
for it (the cheapest that are known to catch it).

A mutant that no pin catches is a hole in the evidence that the oracle
computes the paper's method: the test fails and names it.
"""
import concurrent.futures as cf
import os
import re
import subprocess
import sys
import tempfile

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
P = "tests/test_oracle_pins.py::"
FLUX = "tests/test_oracle_flux.py::test_flux_box_absorption_equals_volume_absorption"
INC = "tests/test_oracle_spectra.py::test_incident_spectrum_and_intensity"

# (name, text in oracle.c, replacement, pins expected to catch it)
MUTANTS = [
    ("C4 enters the E update with the printed + sign (reading 1)",
     "num -= m.C4[p] * En;", "num += m.C4[p] * En;",
     [P + "test_ampere_law_holds_and_pekar"]),
    ("sin(phi) term of C3 with the printed 1/(2 dt Cp) (reading 2)",
     "k.C3[p] = k.C4[p] / 2.0 - EPS0 * A * Om * sin(ph) / (dt * k.Cp[p]);",
     "k.C3[p] = k.C4[p] / 2.0 - EPS0 * A * Om * sin(ph) / (2.0 * dt * k.Cp[p]);",
     [P + "test_critical_point_pole[0.35]"]),
    ("D3 with a factor 2 instead of 4",
     "k.D3 = EPS0 * m->wp * m->wp / (4.0 * k.Dd);", "k.D3 = EPS0 * m->wp * m->wp / (2.0 * k.Dd);",
     [P + "test_local_drude_transverse_wave_recurrence"]),
    ("GNOR: BDF2 history GD^{n-2} dropped from the P_f update",
     "Pn += m.DG1 * gd + m.DG2 * (3.0 * gd - 4.0 * s->GD1[c][q] + s->GD2[c][q]);",
     "Pn += m.DG1 * gd + m.DG2 * (3.0 * gd - 4.0 * s->GD1[c][q]);",
     [P + "test_gnor_longitudinal_plasmon[axis]"]),
    ("grad-div cross difference with a wrong sign",
     "rdP(s, P, b, i, j, k) + rdP(s, P, b, i - w[0], j - w[1], k - w[2]);",
     "rdP(s, P, b, i, j, k) - rdP(s, P, b, i - w[0], j - w[1], k - w[2]);",
     [P + "test_graddiv_is_symmetric_and_negative"]),
    ("curl E: derivative taken along the wrong axis",
     "n1[a1] += 1;", "n1[a2] += 1;",
     [P + "test_vacuum_oblique_plane_wave_matches_discrete_dispersion[1.0-0.5]"]),
    ("curl E with the wrong sign",
     "s->H[c][q] -= s->dt / (MU0 * s->g.dx) * (t1 - t2);", "s->H[c][q] -= s->dt / (MU0 * s->g.dx) * (t2 - t1);",
     [P + "test_vacuum_oblique_plane_wave_matches_discrete_dispersion[1.0-0.5]"]),
    ("E average of f4 weighted (1, 1, 1) instead of (1, 2, 1)",
     "m.D3 * (Em + 2.0 * En + Enext)", "m.D3 * (Em + En + Enext)",
     [P + "test_local_drude_transverse_wave_recurrence"]),
    ("TF/SF conversion of E neighbours with the wrong sign",
     "if (d != 0) v += d * inc_E(s, c, k);", "if (d != 0) v -= d * inc_E(s, c, k);",
     [P + "test_tfsf_no_leakage_without_scatterer[1.0-0.5]"]),
    ("CPML c coefficient with the wrong sign",
     "*c = (sig + alpha) > 0.0 ? sig * (*b - 1.0) / (sig + alpha) : 0.0;",
     "*c = (sig + alpha) > 0.0 ? sig * (1.0 - *b) / (sig + alpha) : 0.0;",
     [P + "test_cpml_normal_incidence_reflection"]),
    ("E_x site placed at the node instead of half a cell along x",
     "static const int E_OFF[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};",
     "static const int E_OFF[3][3] = {{0, 0, 0}, {0, 1, 0}, {0, 0, 1}};",
     [P + "test_voxeliser_brute_force[sphere]"]),
    ("critical points: C2 P_CP^{n-1} term dropped from the E update",
     "num -= (m.C1[p] - 1.0) * s->Pcp[p][c][q] + m.C2[p] * s->Pcpprev[p][c][q];",
     "num -= (m.C1[p] - 1.0) * s->Pcp[p][c][q];",
     [P + "test_ampere_law_holds_and_pekar"]),
    # flux-box assembly and normalisation (the cross sections of Sec. V)
    ("flux: face-edge records weighted 1 instead of 1/2",
     "double w = (idx[other] == lo[other] || idx[other] == hi[other]) ? 0.5 : 1.0;",
     "double w = (idx[other] == lo[other] || idx[other] == hi[other]) ? 1.0 : 1.0;",
     [FLUX]),
    ("flux: H averaged over the two half cells one cell off the face",
     "h[a] = p - 1;", "h[a] = p;",
     [FLUX]),
    ("flux: outward normal of the x faces reversed",
     "double outward = side == 0 ? -1.0 : 1.0;", "double outward = (side == 0) == (a != 0) ? -1.0 : 1.0;",
     [FLUX]),
    ("flux: the -E_c H_b term added instead of subtracted",
     "double tsign = term == 0 ? 1.0 : -1.0;", "double tsign = 1.0;",
     [FLUX]),
    ("flux: H sampled with the phase of n dt instead of (n - 1/2) dt",
     "double tE = s->n * s->dt, tH = (s->n - 0.5) * s->dt;", "double tE = s->n * s->dt, tH = s->n * s->dt;",
     [FLUX]),
    ("flux: face element dx instead of dx^2",
     "double dA = s->g.dx * s->g.dx;", "double dA = s->g.dx;",
     [FLUX]),
    ("flux: absorption taken as the outward (not inward) flux",
     "double sa = -sum[0] * dA / I, ss = sum[1] * dA / I;", "double sa = sum[0] * dA / I, ss = sum[1] * dA / I;",
     [FLUX]),
    # the local Drude model inside the CPML (Sec. III)
    ("nonlocal terms kept inside the CPML",
     "if (m.plasmonic && in_cpml_cell(s, i, j, k)) {", "if (0 && m.plasmonic && in_cpml_cell(s, i, j, k)) {",
     [P + "test_slab_through_the_cpml_stays_bounded"]),
    ("local region of the CPML one cell short",
     "if (ix[a] < s->g.pml || ix[a] >= axis_n(s, a) - s->g.pml) return 1;",
     "if (ix[a] < s->g.pml - 1 || ix[a] >= axis_n(s, a) - s->g.pml) return 1;",
     [P + "test_nonlocal_metal_in_the_cpml_is_local_drude_there"]),
    ("DFT: rectangle rule without the K dt factor",
     "double scale = s->mon.K * s->dt;", "double scale = s->dt;",
     [INC]),
]


def _build(text, d):
    src = os.path.join(d, "oracle.c")
    with open(src, "w") as f:
        f.write(text)
    lib = os.path.join(d, "liboracle.so")
    subprocess.check_call(["gcc", *oracle.GCC_FLAGS, "-I", os.path.join(ROOT, "oracle"), src, "-o", lib, "-lm"])
    return lib


def _run_mutant(m, base):
    name, old, new, pins = m
    with tempfile.TemporaryDirectory() as d:
        lib = _build(base.replace(old, new), d)
        env = dict(os.environ, ORACLE_LIB=lib, OMP_NUM_THREADS="2")
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *pins], cwd=ROOT,
                           env=env, capture_output=True, text=True, timeout=900)
    return name, r.returncode, r.stdout[-2000:]


def test_every_mutation_text_occurs_once():
    base = open(SRC).read()
    for name, old, new, pins in MUTANTS:
        assert base.count(old) == 1, name
        assert old != new


def test_every_planted_mistake_fails_a_pin():
    base = open(SRC).read()
    escaped = []
    with cf.ThreadPoolExecutor(max_workers=max(1, min(4, (os.cpu_count() or 2) // 2))) as ex:
        for name, rc, out in ex.map(lambda m: _run_mutant(m, base), MUTANTS):
            # pytest exits 1 when a test failed; anything else (2: collection
            # or usage error, 5: nothing collected) is not a caught mistake
            if rc != 1 or not re.search(r"\d+ failed", out):
                escaped.append((name, rc, out[-600:]))
    assert not escaped, escaped
