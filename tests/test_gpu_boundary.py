"""Boundary features of the C ABI on the GPU, against the FP64 oracle:
the free-electron charge density as an nlf_get_field target (Eq. Nsol), a
material map handed over in device memory, the flux-record weights getter,
and nlf_sync's bounded wait."""
import numpy as np
import pytest

import oracle
from paper_2005_06997_gb300 import nlfdtd
from paper_2005_06997_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def small_problem():
    prob = W.small_sphere(n=36, steps=0, nf=8, K=4)
    return prob


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_density_field_matches_oracle():
    """div P_f at every node (C/m^3): the GPU's kernel against the oracle's
    backward differences of its FP64 P_f.  The differences of neighbouring
    P_f values cancel most of their magnitude, so the FP32 P_f rounding
    (relative 1e-7 of P_f) is amplified by |P_f| / |div P_f dx|; the bar
    is 1e-4 of the density's norm all the same."""
    prob = small_problem()
    g = nlfdtd.Solver(prob)
    g.run(500)
    g.sync()
    o = oracle.Sim(prob)
    o.step(500)
    got = g.field("density")
    ref = o.density()
    assert np.linalg.norm(ref) > 0
    assert rel_l2(got, ref) <= 1e-4
    # the density lives on the metal: zero well away from it
    assert np.all(got[:4] == 0.0)
    # written to device memory as well
    import torch
    d = torch.empty(got.shape, dtype=torch.float32, device="cuda")
    g.field_to_device("density", d.data_ptr())
    assert np.array_equal(d.cpu().numpy(), got)
    g.close()


def test_device_material_map_equals_shapes():
    """A material map handed over in device memory gives the same voxels and,
    bit for bit, the same fields as the same geometry given as shapes."""
    import torch
    prob = small_problem()
    a = nlfdtd.Solver(prob)
    a.run(300)
    a.sync()
    vox = a.voxels()
    dmap = torch.tensor(vox, device="cuda")
    b = nlfdtd.Solver(prob, material_map=dmap)
    b.run(300)
    b.sync()
    assert np.array_equal(b.voxels(), vox)
    for f in ("Ex", "Hy", "Px", "Pz"):
        assert np.array_equal(a.field(f), b.field(f)), f
    a.close()
    b.close()


def test_flux_weights_follow_the_documented_record_order():
    prob = small_problem()
    g = nlfdtd.Solver(prob)
    coef, n_abs = g.flux_weights()
    rec, coef_o = oracle.Sim(prob).records()
    assert np.array_equal(coef, coef_o)
    assert n_abs == int(np.count_nonzero(rec[:, 0] == 0))
    g.close()


def test_sync_times_out_then_completes():
    """nlf_sync with a zero budget on a long solve reports NLF_E_TIMEOUT and
    loses nothing: waiting again completes the run, equal to one that was
    never interrupted."""
    prob = W.config_sphere_au_gnor_224()
    g = nlfdtd.Solver(prob)
    g.run(2000)
    with pytest.raises(nlfdtd.NLFError) as e:
        g.sync(0)
    assert e.value.code == -7
    g.sync(-1)
    assert g.n == 2000
    ex = g.field("Ex")
    h = nlfdtd.Solver(prob)
    h.run(2000)
    h.sync()
    assert np.array_equal(h.field("Ex"), ex)
    g.close()
    h.close()
