"""The operator held fixed (inner loop of the nested SCF): fock_set_occupied
once, fock_apply_fixed on trial orbitals many times, against the oracle."""

import numpy as np
import pytest

import oracle
from paper_1305_7313_gb300 import FockPlan, _lib, synth
from tests._common import cubic, rel_inf, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(_lib.PREC_FP64, 1e-10), (_lib.PREC_DF64, 1e-10), (_lib.PREC_MIXED32, 2e-5)])
def test_fixed_operator_on_trial_orbitals(prec, tol):
    torch = require_gpu()
    N, L, ecut = 32, 9.0, 12.0
    cell = cubic(L)
    plan = FockPlan(N, cell, ecut, _lib.ERFC, 0.4, prec)
    c = synth.orbitals(plan.miller, cell, 7, 11)
    occ = np.array([2.0, 2.0, 1.5, 1.0, 1.0, 0.5, 0.2])
    psi = torch.from_numpy(c).cuda()
    plan.set_occupied(psi, occ)
    plan.set_batch(3)
    for nt, seed in [(5, 1), (2, 2), (9, 3)]:  # the workspace grows between calls
        t = synth.orbitals(plan.miller, cell, nt, 100 + seed)
        v = plan.apply_fixed(torch.from_numpy(t).cuda()).cpu().numpy()
        vref = oracle.fock_apply_to(c, occ, t, plan.miller, (N, N, N), cell, "erfc", 0.4)
        assert rel_inf(v, vref) <= tol
    # phi = psi gives the apply's V_x psi
    vself = plan.apply_fixed(psi).cpu().numpy()
    vfull, _, _ = plan.apply(psi, occ)
    assert rel_inf(vself, vfull.cpu().numpy()) <= tol
    # the apply replaced the occupied set
    with pytest.raises(_lib.FockError) as err:
        plan.apply_fixed(psi)
    assert err.value.status == 1
    plan.close()
