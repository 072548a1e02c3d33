"""Deterministic accumulation (fock_plan_set_deterministic): V_x psi summed
exactly in 64-bit fixed point, per-pair energies summed in a fixed order.
Results are bitwise identical run to run and for every chain batch, and stay
within the FP64 tolerance of the oracle."""

import numpy as np
import pytest

import oracle
from paper_1305_7313_gb300 import FockPlan, _lib, synth
from tests._common import cubic, rel_inf, require_gpu

pytestmark = pytest.mark.gpu


def case(prec, nb=21, N=48, L=13.5, ecut=12.0, omega=0.3, seed=808):
    torch = require_gpu()
    cell = cubic(L)
    plan = FockPlan(N, cell, ecut, _lib.ERFC, omega, prec)
    c = synth.orbitals(plan.miller, cell, nb, seed)
    occ = np.linspace(2.0, 0.25, nb)
    return torch, plan, c, occ, torch.from_numpy(c).cuda(), cell


@pytest.mark.parametrize("prec", [_lib.PREC_FP64, _lib.PREC_DF64], ids=["fp64", "df64"])
def test_bitwise_reproducible_across_runs_and_chain_batches(prec):
    torch, plan, c, occ, psi, cell = case(prec)
    plan.set_deterministic(True)
    runs = []
    for cb in (5, 5, 19, 3):
        plan.set_batch(cb)
        v, e, d = plan.apply(psi, occ, want_dex=True)
        runs.append((v.clone(), e, d))
    for v, e, d in runs[1:]:
        assert torch.equal(v, runs[0][0])
        assert e == runs[0][1] and d == runs[0][2]
    vref, eref, dref = oracle.fock_apply(c, occ, plan.miller, (48, 48, 48), cell, "erfc", 0.3)
    assert rel_inf(runs[0][0].cpu().numpy(), vref) <= 1e-10
    assert abs(runs[0][1] - eref) <= 1e-10 * abs(eref)
    assert abs(runs[0][2] - dref) <= 1e-10 * abs(dref)
    # the ordinary (atomic) accumulation agrees to rounding
    plan.set_deterministic(False)
    v, e, _ = plan.apply(psi, occ)
    assert rel_inf(v.cpu().numpy(), runs[0][0].cpu().numpy()) <= 1e-12
    plan.close()


def test_deterministic_shards_and_fixed_operator():
    torch, plan, c, occ, psi, cell = case(_lib.PREC_FP64, nb=9, N=24, L=10.0, ecut=10.0)
    plan.set_deterministic(True)
    vfull, efull, _ = plan.apply(psi, occ)
    vsum, esum = 0.0, 0.0
    for s in range(3):
        v, e, _ = plan.apply_shard(psi, occ, s, 3)
        vsum = vsum + v.cpu().numpy()
        esum += e
    assert rel_inf(vsum, vfull.cpu().numpy()) <= 1e-13
    assert abs(esum - efull) <= 1e-13 * abs(efull)
    # fixed operator on trial orbitals, twice: identical and at the oracle
    trial = synth.orbitals(plan.miller, cell, 4, 909)
    phi = torch.from_numpy(trial).cuda()
    plan.set_occupied(psi, occ)
    v1 = plan.apply_fixed(phi).clone()
    v2 = plan.apply_fixed(phi)
    assert torch.equal(v1, v2)
    vref = oracle.fock_apply_to(c, occ, trial, plan.miller, (24, 24, 24), cell, "erfc", 0.3)
    assert rel_inf(v1.cpu().numpy(), vref) <= 1e-10
    plan.close()


def test_deterministic_mode_refused_for_the_mixed_form():
    torch, plan, c, occ, psi, cell = case(_lib.PREC_MIXED32, nb=3, N=24, L=10.0, ecut=10.0)
    with pytest.raises(_lib.FockError):
        plan.set_deterministic(True)
    plan.close()
