"""Every form of the GPU path against the oracle's stored record on the
smallest workload (``tests/golden/oracle_gamma_L10_N24_nb8.txt``: 24^3,
L = 10 bohr, Ecut = 10 Ha, 8 bands, seed 1305, f = 2), with no oracle call:
E_x, dE_x/domega, the norm of every V_x psi_b and sampled coefficients.
Tolerances as in test_gpu_parity.py: 1e-10 in FP64 and double-float; 2e-5 on
V_x psi and 5e-6 on the energies in the mixed form."""

import importlib.util
import os

import numpy as np
import pytest

from paper_1305_7313_gb300 import FockPlan, _lib, synth
from tests._common import cubic, require_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("make_oracle_golden",
                                               os.path.join(HERE, "golden", "make_oracle_golden.py"))
golden = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(golden)

KIND = {"spencer_alavi": (_lib.SPENCER_ALAVI, None), "erfc": (_lib.ERFC, 0.106)}
FORMS = [(_lib.PREC_FP64, 1e-10, 1e-10), (_lib.PREC_DF64, 1e-10, 1e-10), (_lib.PREC_MIXED32, 2e-5, 5e-6)]


@pytest.mark.parametrize("prec,tol_v,tol_e", FORMS, ids=["fp64", "df64", "mixed32"])
@pytest.mark.parametrize("kernel", list(KIND))
def test_every_form_matches_the_stored_oracle_record(prec, tol_v, tol_e, kernel):
    torch = require_gpu()
    with open(golden.FILE) as fh:
        rec = golden.parse(fh.read())[kernel]
    cell = cubic(golden.L)
    kind, omega = KIND[kernel]
    plan = FockPlan(golden.N, cell, golden.ECUT, kind, omega, prec)
    c = synth.orbitals(plan.miller, cell, golden.NB, golden.SEED)
    vpsi, ex, dex = plan.apply(torch.from_numpy(c).cuda(), np.full(golden.NB, 2.0),
                               want_dex=omega is not None)
    v = vpsi.cpu().numpy()
    assert abs(ex - rec["ex"]) <= tol_e * abs(rec["ex"])
    if rec["dex"] not in (None, 0.0):
        assert abs(dex - rec["dex"]) <= tol_e * abs(rec["dex"])
    vmax = max(abs(z) for z in rec["coef"].values())
    for b, nrm in rec["norm"].items():
        assert abs(np.linalg.norm(v[b]) - nrm) <= tol_v * nrm
    for (b, g), z in rec["coef"].items():
        assert abs(v[b, g] - z) <= tol_v * vmax
    plan.close()
