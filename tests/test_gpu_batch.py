"""Batched stepping (nlf_batch_run): many uneven grids advanced by one launch
per kernel per time step over their joint work list, against the same grids
run alone and against the oracle."""
import copy
import math

import numpy as np
import pytest

import oracle
from paper_2005_06997_gb300 import nlfdtd
from paper_2005_06997_gb300 import workloads as W

pytestmark = pytest.mark.gpu

VECTORS = {"E": ("Ex", "Ey", "Ez"), "H": ("Hx", "Hy", "Hz"), "P": ("Px", "Py", "Pz")}


def vec_err(a_fields, b_fields):
    out = {}
    for vec, comps in VECTORS.items():
        num = math.sqrt(sum(np.sum((a_fields[c].astype(np.float64) - b_fields[c]) ** 2) for c in comps))
        den = math.sqrt(sum(np.sum(np.asarray(b_fields[c], dtype=np.float64) ** 2) for c in comps))
        out[vec] = num / den if den > 0 else num
    return out


def fields(s):
    return {c: s.field(c) for comps in VECTORS.values() for c in comps}


def instances(n, steps, nf=16):
    out = []
    for p in W.batched_instances(n=n, nf=nf, steps=steps):
        q = copy.deepcopy(p)
        src = W.gaussian_source(q["source"]["tf_lo"], q["source"]["tf_hi"], (1.0, 9.0))
        src["t0"] = 2.5 * src["tau"]
        q["source"] = src
        out.append(q)
    return out


def test_batched_equals_alone_uneven_grids_and_steps():
    probs = instances(6, 0)
    steps = [700, 700, 520, 777, 300, 1100]
    alone = []
    for p, n in zip(probs, steps):
        s = nlfdtd.Solver(p)
        s.run(n)
        s.sync()
        alone.append((fields(s), s.spectra()))
    batch = [nlfdtd.Solver(p) for p in probs]
    status = nlfdtd.batch_run(batch, steps)
    assert status == [0] * len(batch)
    for s, n, (f_alone, sp_alone) in zip(batch, steps, alone):
        s.sync()
        assert s.n == n
        errs = vec_err(fields(s), f_alone)
        assert max(errs.values()) <= 1e-5, errs
        sp = s.spectra()
        for key in ("ext", "abs", "sca"):
            ref = sp_alone[key]
            assert np.max(np.abs(sp[key] - ref)) <= 1e-4 * np.max(np.abs(ref)) + 1e-30, key
    # every batched instance really went through batched launches
    assert sum(s.launches for s in batch) > 0


def test_batched_instance_matches_oracle():
    probs = instances(3, 0, nf=8)
    batch = [nlfdtd.Solver(p) for p in probs]
    steps = [512, 512, 512]
    assert nlfdtd.batch_run(batch, steps) == [0, 0, 0]
    for p, s in zip(probs, batch):
        s.sync()
        o = oracle.Sim(p)
        o.step(512)
        ref = {c: o.array(c) for comps in VECTORS.values() for c in comps}
        errs = vec_err(fields(s), ref)
        assert max(errs.values()) <= 1e-4, errs


def test_unstable_instance_is_isolated():
    """Poison one instance's state with a NaN (through a checkpoint, on the
    host): it reports NLF_E_UNSTABLE, the others match a batch without it
    (to rounding: the autotuner may split the work differently)."""
    probs = instances(3, 0, nf=8)
    ref = [nlfdtd.Solver(p) for p in probs]
    assert nlfdtd.batch_run(ref, [512] * 3) == [0, 0, 0]
    ref_f = [fields(s) for s in ref]
    runs = [nlfdtd.Solver(p) for p in probs]
    bad = runs[1]
    snap = bad.save_state()
    # the E_x arrays start 256 bytes into the state (after the header): poison one value
    view = snap.view(np.float32)
    view[64 + 1000] = np.nan
    bad.load_state(snap)
    nlfdtd.batch_run(runs, [512] * 3)
    with pytest.raises(nlfdtd.NLFError) as ei:
        bad.sync()
    assert ei.value.code == -6
    for q in (0, 2):
        runs[q].sync()
        errs = vec_err(fields(runs[q]), ref_f[q])
        assert max(errs.values()) <= 1e-6, (q, errs)


def edge_instances():
    """Geometries at the edges of the tiling and the TF/SF surface: a grid
    narrower than one tile with the TF surface one cell from every PEC wall,
    a CPML on one axis beside PEC walls with a one-plane z chunk, and a
    dielectric background at another Courant number."""
    def early(q):
        src = W.gaussian_source(q["source"]["tf_lo"], q["source"]["tf_hi"], (1.0, 9.0))
        src["t0"] = 2.5 * src["tau"]
        q["source"] = src
        return q

    out = []
    q = W.small_sphere(n=36, steps=0, nf=4, K=4)
    q.update(shape=(13, 11, 18), pml=0, bc=("pec",) * 3, monitors=None,
             shapes=[W.sphere_shape((13, 8, 18), 2, 1)])
    q["source"]["tf_lo"], q["source"]["tf_hi"] = (1, 1, 1), (12, 10, 17)
    out.append(early(q))
    q = W.small_sphere(n=36, steps=0, nf=4, K=4)
    q.update(shape=(40, 44, 17), pml=6, bc=("pec", "cpml", "pec"), monitors=None,
             shapes=[W.sphere_shape((40, 44, 17), 6, 1)])
    q["source"]["tf_lo"], q["source"]["tf_hi"] = (2, 7, 2), (37, 36, 14)
    out.append(early(q))
    q = W.small_sphere(n=36, steps=0, nf=4, K=4)
    q["eps_b"], q["courant"], q["monitors"] = 1.77, 0.45, None
    out.append(early(q))
    return out


def test_batched_edge_geometries_match_oracle():
    probs = edge_instances()
    batch = [nlfdtd.Solver(p) for p in probs]
    steps = [400, 400, 400]
    assert nlfdtd.batch_run(batch, steps) == [0, 0, 0]
    for p, s in zip(probs, batch):
        s.sync()
        o = oracle.Sim(p)
        o.step(400)
        ref = {c: o.array(c) for comps in VECTORS.values() for c in comps}
        errs = vec_err(fields(s), ref)
        assert max(errs.values()) <= 1e-4, (p["shape"], errs)


def _busy_copy_engines(torch, side, mb=256, rounds=8):
    """Queue `rounds` pinned host-to-device copies of `mb` MB on stream `side`
    (keeps the copy engines busy while other streams launch work)."""
    host = torch.empty(mb << 20, dtype=torch.uint8).pin_memory()
    dev = torch.empty(mb << 20, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(side):
        for _ in range(rounds):
            dev.copy_(host, non_blocking=True)
    return host, dev


def test_batched_plans_on_a_non_blocking_stream_with_busy_copy_engines():
    """Batched plans made and launched on a non-blocking stream (a torch
    stream, as the server's lanes use) while another stream keeps the copy
    engines busy: every new plan's descriptors are on the device before its
    first launch, so the fields equal those of the same batch on the legacy
    default stream.  The member set shrinks every DFT period, so each period
    makes a new plan."""
    torch = pytest.importorskip("torch")
    probs = instances(4, 0, nf=8)
    b = 8
    U = 16 * b
    steps = [4 * U, 3 * U, 2 * U, U]
    ref = [nlfdtd.Solver(p, block_b=b) for p in probs]
    assert nlfdtd.batch_run(ref, steps) == [0] * 4
    ref_f = [fields(s) for s in ref]
    runs = [nlfdtd.Solver(p, block_b=b) for p in probs]
    lane, side = torch.cuda.Stream(), torch.cuda.Stream()
    keep = _busy_copy_engines(torch, side)
    status = nlfdtd.batch_run(runs, steps, lane.cuda_stream)
    side.synchronize()
    del keep
    assert status == [0] * 4
    for q, (s, f) in enumerate(zip(runs, ref_f)):
        s.sync()
        assert s.n == steps[q]
        errs = vec_err(fields(s), f)
        assert max(errs.values()) <= 1e-6, (q, errs)


def test_state_and_field_writes_land_before_a_run_on_a_non_blocking_stream():
    """nlf_load_state and nlf_set_field copy on the context's stream (here
    the legacy default stream) and wait: a run launched right after on a
    non-blocking stream, with the copy engines busy, starts from the loaded
    state and the set field."""
    torch = pytest.importorskip("torch")
    p = instances(1, 0, nf=8)[0]
    a = nlfdtd.Solver(p)
    a.run(300)
    a.sync()
    snap = a.save_state()
    ex = a.field("Ex")
    a.run(200)
    a.sync()
    ref = fields(a)
    lane, side = torch.cuda.Stream(), torch.cuda.Stream()
    s = nlfdtd.Solver(p)
    s.run(0)                                   # state initialised on the legacy stream
    keep = _busy_copy_engines(torch, side)
    s.load_state(snap)
    s.run(200, lane.cuda_stream)
    s.sync()
    side.synchronize()
    errs = vec_err(fields(s), ref)
    assert max(errs.values()) <= 1e-7, errs
    # the same with E_x written over the loaded state: a changed field is seen
    c = nlfdtd.Solver(p)
    c.run(0)
    c.load_state(snap)
    c.set_field("Ex", 2.0 * ex)
    c.run(200)
    c.sync()
    ref2 = fields(c)
    t = nlfdtd.Solver(p)
    t.run(0)
    t.load_state(snap)
    keep2 = _busy_copy_engines(torch, side)
    t.set_field("Ex", 2.0 * ex)
    t.run(200, lane.cuda_stream)
    t.sync()
    side.synchronize()
    del keep, keep2
    errs = vec_err(fields(t), ref2)
    assert max(errs.values()) <= 1e-7, errs
    assert vec_err(ref2, ref)["E"] > 1e-3          # the set field changed the run
