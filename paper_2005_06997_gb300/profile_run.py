"""Run a named workload for a few time steps (the command that profiles are
taken on: ``python -m paper_2005_06997_gb300.profile_run <workload> <steps> [nf]``).

It configures the problem through the C ABI, runs `steps` time steps, reads
the spectra and prints the launch count.  The kernels and the problem are the
benchmark's; only the number of time steps and, if given, the number of DFT
frequencies (every nf-th of the 200, to keep a profiler's memory save/restore
small; the time-step kernel does not depend on it) differ.
"""
import sys

import torch

from . import nlfdtd
from . import workloads as W


def main():
    name = sys.argv[1] if len(sys.argv) > 1 else "sphere_au_gnor_r10nm_224"
    steps = int(sys.argv[2]) if len(sys.argv) > 2 else 20
    torch.cuda.set_device(0)
    prob = W.CONFIGS[name]()
    if len(sys.argv) > 3:
        nf = int(sys.argv[3])
        om = prob["monitors"]["omega"]
        prob["monitors"]["omega"] = om[:: max(1, len(om) // nf)][:nf]
    s = nlfdtd.Solver(prob)
    s.run(steps)
    s.sync()
    spec = s.spectra()
    print("%s: %d steps, %d kernel launches, state %.2f GB, finite spectra %s" %
          (name, steps, s.launches, s.state_bytes() / 1e9, bool((spec["ext"] == spec["ext"]).all())))


if __name__ == "__main__":
    main()
