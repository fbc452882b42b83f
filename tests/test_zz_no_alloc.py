"""nlf_flux_spectra_static: cross sections from caller-held accumulators with
the partial sums in the library's fixed device array (no allocation), against
nlf_get_spectra on the same run, on two calls in a row.

The accumulators come from nlf_get_dft and the face weights from the oracle's
record list (the same documented record order), both copied into the caller's
own device memory, as a caller without cudaMalloc would hold them.  This file
is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2005_06997_gb300 import nlfdtd
from paper_2005_06997_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_scratch_spectra_match_context_spectra():
    import torch
    prob = W.small_sphere(n=36, steps=0, nf=24, K=4, band_ev=(1.5, 8.5))
    src = W.gaussian_source(prob["source"]["tf_lo"], prob["source"]["tf_hi"], (1.5, 8.5))
    src["t0"] = 2.5 * src["tau"]
    prob["source"] = src
    s = nlfdtd.Solver(prob)
    s.run(1200)
    ref = s.spectra()                                  # existing entry point (context scratch)
    aE, aH = s.dft()
    rec, coef = oracle.Sim(prob).records()
    nrec = len(coef)
    assert aE.shape[0] == nrec + 1
    n_abs = int(np.count_nonzero(rec[:, 0] == 0))
    nf = aE.shape[1]
    dev = torch.device("cuda")
    t_e = torch.tensor(np.ascontiguousarray(aE), dtype=torch.float64, device=dev)
    t_h = torch.tensor(np.ascontiguousarray(aH), dtype=torch.float64, device=dev)
    t_c = torch.tensor(np.ascontiguousarray(coef), dtype=torch.float64, device=dev)
    L = nlfdtd.load()
    outs = []
    for _ in range(2):
        out = torch.full((4 * nf,), float("nan"), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream()
        rc = L.nlf_flux_spectra_static(ctypes.c_void_p(t_e.data_ptr()), ctypes.c_void_p(t_h.data_ptr()),
                                       ctypes.c_void_p(t_c.data_ptr()), n_abs, nrec, nf, prob["dx"] ** 2,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    for o in outs:
        for q, key in enumerate(("ext", "abs", "sca")):
            got = o[q * nf:(q + 1) * nf]
            want = ref[key]
            assert np.max(np.abs(got - want)) <= 1e-9 * np.max(np.abs(want)), key
    assert np.array_equal(outs[0], outs[1])
    # sizes beyond the static array are rejected before any launch
    rc = L.nlf_flux_spectra_static(ctypes.c_void_p(t_e.data_ptr()), ctypes.c_void_p(t_h.data_ptr()),
                                   ctypes.c_void_p(t_c.data_ptr()), n_abs, nrec, 155649,
                                   prob["dx"] ** 2, ctypes.c_void_p(t_e.data_ptr()), None)
    assert rc == -1
