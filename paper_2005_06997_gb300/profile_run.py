"""Run a named workload for a few time steps (the command that profiles are
taken on: ``python -m paper_2005_06997_gb300.profile_run <workload> <steps> [nf]
[pec] [nosource] [nometal]``).

It configures the problem through the C ABI, runs `steps` time steps, reads
the spectra and prints the launch count.  The name ``batched64`` runs the
64-instance batched configuration through nlf_batch_run instead.  The kernels and the problem are the
benchmark's; only the number of time steps and, if given, the number of DFT
frequencies (every nf-th of the 200, to keep a profiler's memory save/restore
small; the time-step kernel does not depend on it) differ.  The words pec,
nosource and nometal select the same grid with PEC walls instead of the CPML,
without the TF/SF source and monitors, or without the particle.
"""
import sys

import torch

from . import nlfdtd
from . import workloads as W


def run_batched(n, steps):
    """The seeded batched configuration (n sphere / dimer solves on uneven
    grids) advanced together by nlf_batch_run for `steps` time steps."""
    solvers = [nlfdtd.Solver(p) for p in W.batched_instances(n=n)]
    try:
        status = nlfdtd.batch_run(solvers, [steps] * n)
        for s in solvers:
            s.sync()
        launches = sum(s.launches for s in solvers)
        cells = sum(s.info()["cells"] for s in solvers)
        print("batched %d instances: %d steps, status %s, %d kernel launches counted over the contexts, %.1f M cells"
              % (n, steps, "ok" if not any(status) else status, launches, cells / 1e6))
    finally:
        for s in solvers:
            s.close()


def main():
    name = sys.argv[1] if len(sys.argv) > 1 else "sphere_au_gnor_r10nm_224"
    steps = int(sys.argv[2]) if len(sys.argv) > 2 else 20
    torch.cuda.set_device(0)
    if name == "batched64":
        run_batched(64, steps)
        return
    prob = W.CONFIGS[name]()
    if len(sys.argv) > 3:
        nf = int(sys.argv[3])
        om = prob["monitors"]["omega"]
        prob["monitors"]["omega"] = om[:: max(1, len(om) // nf)][:nf]
    words = set(sys.argv[4:])
    if "pec" in words:
        prob["bc"] = ("pec",) * 3
    if "nosource" in words:
        prob["source"] = None
        prob["monitors"] = None
    if "nometal" in words:
        prob["shapes"] = []
    s = nlfdtd.Solver(prob)
    s.run(steps)
    s.sync()
    fin = None
    if prob.get("monitors") is not None:
        spec = s.spectra()
        fin = bool((spec["ext"] == spec["ext"]).all())
    print("%s %s: %d steps, %d kernel launches, state %.2f GB, finite spectra %s" %
          (name, " ".join(sorted(words)), steps, s.launches, s.state_bytes() / 1e9, fin))


if __name__ == "__main__":
    main()
