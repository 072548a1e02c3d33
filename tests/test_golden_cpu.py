"""The oracle reproduces its stored record on the smallest workload
(``tests/golden/oracle_gamma_L10_N24_nb8.txt``, written by
``tests/golden/make_oracle_golden.py``): a change to the oracle's arithmetic
shows up here and must name the passage of the paper that justifies it."""

import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("make_oracle_golden",
                                               os.path.join(HERE, "golden", "make_oracle_golden.py"))
golden = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(golden)

RTOL = 1e-12  # FP64 rounding of a different FFT library build, far below any physics


def test_the_oracle_reproduces_its_stored_record():
    with open(golden.FILE) as fh:
        rec = golden.parse(fh.read())
    npw, out = golden.compute()
    assert npw == rec["npw"] == 1503
    for kind, _ in golden.KERNELS:
        v, ex, dex = out[kind]
        r = rec[kind]
        assert abs(ex - r["ex"]) <= RTOL * abs(r["ex"])
        if r["dex"] not in (None, 0.0):
            assert abs(dex - r["dex"]) <= RTOL * abs(r["dex"])
        vmax = max(abs(z) for z in r["coef"].values())
        for b, nrm in r["norm"].items():
            assert abs(np.linalg.norm(v[b]) - nrm) <= RTOL * nrm
        for (b, g), z in r["coef"].items():
            assert abs(v[b, g] - z) <= RTOL * vmax
