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


def test_the_oracle_reproduces_one_band_of_the_full_size_record():
    # tests/golden/oracle_fullsize_N96_nb64.txt (96^3, first 64 bands): V_x psi
    # of one sampled band per case, recomputed by the oracle over the same 64
    # source bands (64 ordered pairs, seconds); the stored E_x values are the
    # same run's sums over all 64 x 64 pairs
    import oracle
    from tests.golden import fullsize_record
    spec = importlib.util.spec_from_file_location("make_fullsize_golden",
                                                  os.path.join(HERE, "golden", "make_fullsize_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    rec = fullsize_record.load()
    cell = (mk.L * np.eye(3)).ravel()
    grid = (mk.N, mk.N, mk.N)
    mill, _ = oracle.gsphere(grid, cell, mk.ECUT)
    assert len(mill) == rec["npw"] == 39127 and rec["nb"] == mk.NB == 64
    for (name, kind, omega, seed), band in zip(mk.CASES, (0, 63)):
        r = rec[name]
        assert r["ex"] < 0 and (r["dex"] == 0.0) == (omega is None)
        c = mk.synth.orbitals(mill, cell, mk.NB_ALL, seed)[:mk.NB]
        v, _, _ = oracle.fock_apply(c, np.full(mk.NB, 2.0), mill, grid, cell, kind, omega, out_bands=[band])
        assert abs(np.max(np.abs(v[0])) - r["vmax"][band]) <= RTOL * r["vmax"][band]
        for (b, g), z in r["coef"].items():
            if b == band:
                assert abs(v[0, g] - z) <= RTOL * r["vmax"][band]
