"""Brillouin-zone-sampled apply (complex periodic parts, v(G + q)) against the
FP64 k-point oracle."""

import numpy as np
import pytest

import oracle
from paper_1305_7313_gb300 import FockKPlan, _lib, synth
from tests._common import cubic, rel_inf, require_gpu

pytestmark = pytest.mark.gpu

KPTS = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.0, 0.5, 0.5], [0.25, -0.25, 0.5]])
WK = np.array([0.4, 0.2, 0.3, 0.1])


def kcase(N, L, ecut, nb, kind, omega, prec, kpts=KPTS, wk=WK, seed=40):
    torch = require_gpu()
    cell = cubic(L)
    plan = FockKPlan(N, cell, ecut, kpts, wk, kind, omega, prec)
    cs, mills, psi = [], [], []
    for k in range(len(kpts)):
        m = plan.miller(k)
        mo, _ = oracle.gsphere_k((N, N, N), cell, ecut, kpts[k])
        assert np.array_equal(m, mo)
        c = synth.orbitals_k(m, cell, kpts[k], nb, seed + k)
        cs.append(c)
        mills.append(m)
        psi.append(torch.from_numpy(c).cuda())
    occ = np.linspace(2.0, 0.5, nb)[None, :].repeat(len(kpts), 0)
    return torch, plan, cs, mills, psi, occ, cell


@pytest.mark.parametrize("prec,tol_v,tol_e", [(_lib.PREC_FP64, 1e-10, 1e-10), (_lib.PREC_MIXED32, 2e-5, 5e-6)])
def test_kpoints_match_the_oracle(prec, tol_v, tol_e):
    # 16^3 at L = 7, Ecut = 4: the pair densities of the four spheres reach
    # frequency differences of 6 < 8, so no pair reaches the Nyquist plane
    N = 16
    torch, plan, cs, mills, psi, occ, cell = kcase(N, 7.0, 4.0, 3, _lib.ERFC, 0.5, prec)
    plan.set_batch(4)  # several pair launches, ragged tail
    vk, ex = plan.apply(psi, occ)
    vref, eref = oracle.fock_apply_kpoints(cs, occ, mills, KPTS, WK, (N, N, N), cell, "erfc", 0.5)
    assert abs(ex - eref) <= tol_e * abs(eref)
    vmax = max(np.max(np.abs(v)) for v in vref)
    for k in range(len(KPTS)):
        assert np.max(np.abs(vk[k].cpu().numpy() - vref[k])) <= tol_v * vmax


def test_gamma_only_complex_orbitals_match_the_gamma_oracle():
    # Ecut 6 at L = 10: the pair densities reach |m| = 10 < 12
    N = 24
    kp = np.zeros((1, 3))
    torch, plan, cs, mills, psi, occ, cell = kcase(N, 10.0, 6.0, 5, _lib.SPENCER_ALAVI, None, _lib.PREC_FP64,
                                                    kpts=kp, wk=[1.0])
    vk, ex = plan.apply(psi, occ)
    vref, eref, _ = oracle.fock_apply(cs[0], occ[0], mills[0], (N, N, N), cell, "spencer_alavi", real=False)
    assert abs(ex - eref) <= 1e-10 * abs(eref)
    assert rel_inf(vk[0].cpu().numpy(), vref) <= 1e-10


@pytest.mark.parametrize("prec,tol_v,tol_e", [(_lib.PREC_FP64, 1e-10, 1e-10), (_lib.PREC_MIXED32, 2e-5, 5e-6)])
def test_two_k_points_spencer_alavi_several_launches(prec, tol_v, tol_e):
    # 2 k points x 6 bands: 78 unique pairs in launches of 5 chains (ragged tail of 3)
    N = 24
    kp = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    wk = np.array([0.75, 0.25])
    torch, plan, cs, mills, psi, occ, cell = kcase(N, 9.0, 8.0, 6, _lib.SPENCER_ALAVI, None, prec, kpts=kp,
                                                    wk=wk, seed=90)
    plan.set_batch(5)
    vk, ex = plan.apply(psi, occ)
    vref, eref = oracle.fock_apply_kpoints(cs, occ, mills, kp, wk, (N, N, N), cell, "spencer_alavi")
    assert abs(ex - eref) <= tol_e * abs(eref)
    vmax = max(np.max(np.abs(v)) for v in vref)
    for k in range(2):
        assert np.max(np.abs(vk[k].cpu().numpy() - vref[k])) <= tol_v * vmax


def test_one_band_per_k_point_and_empty_bands():
    # nb = 1 (only pairs across k points and self pairs), then a zero occupation
    N = 16
    torch, plan, cs, mills, psi, occ, cell = kcase(N, 7.0, 4.0, 1, _lib.ERFC, 0.5, _lib.PREC_FP64, seed=120)
    vk, ex = plan.apply(psi, occ)
    vref, eref = oracle.fock_apply_kpoints(cs, occ, mills, KPTS, WK, (N, N, N), cell, "erfc", 0.5)
    assert abs(ex - eref) <= 1e-10 * abs(eref)
    vmax = max(np.max(np.abs(v)) for v in vref)
    for k in range(len(KPTS)):
        assert np.max(np.abs(vk[k].cpu().numpy() - vref[k])) <= 1e-10 * vmax
    occ0 = occ.copy()
    occ0[1, 0] = 0.0
    vk, ex = plan.apply(psi, occ0)
    vref, eref = oracle.fock_apply_kpoints(cs, occ0, mills, KPTS, WK, (N, N, N), cell, "erfc", 0.5)
    assert abs(ex - eref) <= 1e-10 * abs(eref)
    for k in range(len(KPTS)):
        assert np.max(np.abs(vk[k].cpu().numpy() - vref[k])) <= 1e-10 * vmax


def test_aliasing_grid_is_refused_and_the_device_stays_usable():
    # 16^3 at L = 7, Ecut = 6: frequency differences reach 8 = N/2; the plan is
    # refused on the host, then a plan on a grid that holds the pair densities
    # runs and matches the oracle
    require_gpu()
    with pytest.raises(_lib.FockError) as e:
        FockKPlan(16, cubic(7.0), 6.0, KPTS, WK, _lib.ERFC, 0.5, _lib.PREC_FP64)
    assert e.value.status == 3 and "Nyquist" in str(e.value)
    N = 24
    kp = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    torch, plan, cs, mills, psi, occ, cell = kcase(N, 7.0, 6.0, 2, _lib.ERFC, 0.5, _lib.PREC_FP64, kpts=kp,
                                                    wk=[0.5, 0.5], seed=140)
    vk, ex = plan.apply(psi, occ)
    vref, eref = oracle.fock_apply_kpoints(cs, occ, mills, kp, [0.5, 0.5], (N, N, N), cell, "erfc", 0.5)
    assert abs(ex - eref) <= 1e-10 * abs(eref)
    vmax = max(np.max(np.abs(v)) for v in vref)
    for k in range(2):
        assert np.max(np.abs(vk[k].cpu().numpy() - vref[k])) <= 1e-10 * vmax


@pytest.mark.parametrize("kind,omega", [(_lib.SPENCER_ALAVI, None), (_lib.ERFC, 0.5)], ids=["sa", "erfc"])
def test_mixed_kpoints_take_the_g0_term_from_fp64_overlaps(kind, omega):
    # one k point (q = 0 for its pairs), one state whose periodic part is a
    # constant (c = 1 at G = 0): the pair density is constant, its transform
    # vanishes away from G = 0 in any arithmetic, and the one kernel term
    # comes from the FP64 overlap and the FP64 table: E_x to FP64 rounding
    # (the FP32 transform's own value is good to ~1e-7 only)
    torch = require_gpu()
    N, L, ecut = 16, 7.0, 4.0
    kp = np.array([[0.5, 0.0, 0.0]])
    cell = cubic(L)
    plan = FockKPlan(N, cell, ecut, kp, [1.0], kind, omega, _lib.PREC_MIXED32)
    m = plan.miller(0)
    c = np.zeros((1, len(m)), dtype=np.complex128)
    c[0, int(np.flatnonzero(np.all(m == 0, axis=1))[0])] = 1.0
    occ = np.array([[2.0]])
    _, ex = plan.apply([torch.from_numpy(c).cuda()], occ)
    ok = "spencer_alavi" if kind == _lib.SPENCER_ALAVI else "erfc"
    _, eref = oracle.fock_apply_kpoints([c], occ, [m], kp, [1.0], (N, N, N), cell, ok, omega)
    assert abs(ex - eref) <= 1e-13 * abs(eref)
