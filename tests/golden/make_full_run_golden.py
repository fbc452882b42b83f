#!/usr/bin/env python3
"""Write the FP64 oracle's results for a full-length run of a named workload.

    python tests/golden/make_full_run_golden.py sphere_au_gnor_r10nm_224
    python tests/golden/make_full_run_golden.py cube_tips_au_gnor_512_pulse

Calls only ``oracle/`` (and the seeded problem descriptions of
``paper_2005_06997_gb300.workloads``, which hold no method arithmetic).  The
run is the workload as configured (grid, material, source, monitors, number
of time steps).  Stored in ``tests/golden/full_run_<workload>.npz``:

  spectra      ext, abs, sca [m^2] and the incident intensity I over the
               workload's frequencies (the absorption / scattering /
               extinction cross sections of Sec. V);
  sumsq_*      the sum of squares of every field component after the run
               (E in V/m, H in A/m, P_f in C/m^2);
  idx_*, val_* seeded sample sites (flat [nz][ny][nx] indices) and the
               oracle's values there: for each E and H component 1024 sites
               over the whole grid and 1024 inside the particle's bounding
               box, for each P_f component 1024 plasmonic sites;
  rec_idx, dftE, dftH  the raw DFT accumulators (SI, K dt included) of 16
               seeded flux records and of the incident record (last row).

The samples are drawn with numpy.random.default_rng(20050697) from sizes
alone, so the GPU test draws the same sites without running the oracle.

A pulse run (workloads.pulse_run: a workload's grid and particle without
source and monitors, started from a divergence-free pulse) stores the field
entries only; its sample box is the particle's bounding box.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2005_06997_gb300 import workloads as W  # noqa: E402

SEED = 20050697
N_GRID = 1024
N_BOX = 1024
N_METAL = 1024
N_REC = 16


def sample_sites(shape3, box_lo, box_hi, metal_flat, nrec):
    """Seeded sample sites: (grid, box) indices per E/H component, metal
    indices per P component, and flux-record indices.  metal_flat[c] lists
    the flat indices of the plasmonic sites of component c (sorted)."""
    rng = np.random.default_rng(SEED)
    nz, ny, nx = shape3
    out = {}
    for name in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz"):
        g = rng.integers(0, nx * ny * nz, size=N_GRID)
        bi = rng.integers(box_lo[0], box_hi[0] + 1, size=N_BOX)
        bj = rng.integers(box_lo[1], box_hi[1] + 1, size=N_BOX)
        bk = rng.integers(box_lo[2], box_hi[2] + 1, size=N_BOX)
        b = (bk * ny + bj) * nx + bi
        out[name] = np.concatenate([g, b]).astype(np.int32)
    for c, name in enumerate(("Px", "Py", "Pz")):
        m = metal_flat[c]
        out[name] = m[rng.integers(0, len(m), size=N_METAL)].astype(np.int32)
    out["rec"] = np.sort(rng.choice(nrec, size=N_REC, replace=False)).astype(np.int32)
    return out


def particle_box(prob):
    """Cells of the absorption box (the particle with its margin)."""
    mo = prob["monitors"]
    return tuple(mo["abs_lo"]), tuple(mo["abs_hi"])


def metal_box(vox):
    """Inclusive cell bounds (x, y, z) of every E-site that holds a material."""
    any_m = (vox[0] != 0) | (vox[1] != 0) | (vox[2] != 0)
    ks, js, is_ = (np.flatnonzero(any_m.any(axis=a)) for a in ((1, 2), (0, 2), (0, 1)))
    return (int(is_[0]), int(js[0]), int(ks[0])), (int(is_[-1]), int(js[-1]), int(ks[-1]))


def main():
    name = sys.argv[1] if len(sys.argv) > 1 else "sphere_au_gnor_r10nm_224"
    pulse = name not in W.CONFIGS
    if pulse:
        prob, (ex, ey), steps = W.pulse_run(name)
    else:
        prob = W.CONFIGS[name]()
        steps = int(prob["steps"])
    t0 = time.time()
    s = oracle.Sim(prob)
    if pulse:
        s.array("Ex")[...] = ex
        s.array("Ey")[...] = ey
        del ex, ey
    done = 0
    chunk = 256
    while done < steps:
        k = min(chunk, steps - done)
        s.step(k)
        done += k
        print("%s: %d / %d steps, %.0f s" % (name, done, steps, time.time() - t0), flush=True)
    spec = None if pulse else s.spectra()
    vox = s.material_map()
    metal_flat = []
    for c in range(3):
        plas = np.zeros(vox[c].size, dtype=bool)
        for q, m in enumerate(prob["materials"]):
            if m.get("wp", 0.0) > 0.0:
                plas |= vox[c].reshape(-1) == q + 1
        metal_flat.append(np.flatnonzero(plas))
    lo, hi = metal_box(vox) if pulse else particle_box(prob)
    smp = sample_sites(s.shape3, lo, hi, metal_flat, 64 if pulse else s.nrec)
    out = {} if pulse else {"ext": spec["ext"], "abs": spec["abs"], "sca": spec["sca"], "inc": spec["inc"]}
    for fname in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "Px", "Py", "Pz"):
        a = np.asarray(s.array(fname), dtype=np.float64).reshape(-1)
        out["sumsq_" + fname] = np.array(float(np.sum(a * a)))
        out["idx_" + fname] = smp[fname]
        out["val_" + fname] = a[smp[fname]]
    if not pulse:
        aE, aH = s.dft()
        rows = np.concatenate([smp["rec"], [s.nrec]]).astype(np.int32)
        out["rec_idx"] = rows
        out["dftE"] = aE[rows]
        out["dftH"] = aH[rows]
    try:
        rev = subprocess.run(["git", "-C", ROOT, "rev-parse", "--short", "HEAD"], capture_output=True,
                             text=True).stdout.strip()
    except Exception:
        rev = "unknown"
    meta = {"workload": name, "steps": steps, "seed": SEED, "oracle_commit": rev,
            "command": "python tests/golden/make_full_run_golden.py %s" % name,
            "wall_s": time.time() - t0, "threads": os.environ.get("OMP_NUM_THREADS", "all")}
    out["meta"] = np.array(json.dumps(meta))
    path = os.path.join(HERE, "full_run_%s.npz" % name)
    np.savez_compressed(path, **out)
    print("wrote", path, meta, flush=True)
    s.close()


if __name__ == "__main__":
    main()
