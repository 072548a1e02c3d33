"""E_x(psi, omega) as a torch.autograd.Function: gradients against central
finite differences (FP64 form), the FP64 oracle's gradient, and the mixed form
against the FP64 form.  Workload: 72^3 grid, L = 20 bohr, Ecut = 12 Ha,
256 bands, erfc kernel with omega = 0.106."""

import numpy as np
import pytest

import oracle
from paper_1305_7313_gb300 import _lib, synth
from paper_1305_7313_gb300.autograd import exchange_energy
from tests._common import cubic, rel_inf, require_gpu

pytestmark = pytest.mark.gpu

N, L, ECUT, NB, OMEGA = 72, 20.0, 12.0, 256, 0.106


@pytest.fixture(scope="module")
def case():
    torch = require_gpu()
    cell = cubic(L)
    mill, _ = oracle.gsphere((N, N, N), cell, ECUT)
    c = synth.orbitals(mill, cell, NB, 1309)
    return dict(torch=torch, cell=cell, mill=mill, c=c, occ=np.full(NB, 2.0))


def energy_and_grads(case, c, omega, prec, occ=None):
    torch = case["torch"]
    psi = torch.from_numpy(c).cuda().requires_grad_(True)
    om = torch.tensor(omega, dtype=torch.float64, requires_grad=True)
    e = exchange_energy(psi, case["occ"] if occ is None else occ, N, case["cell"], ECUT,
                        _lib.ERFC, om, prec)
    e.backward()
    return float(e.detach().cpu()), psi.grad.detach().cpu().numpy(), float(om.grad)


def test_gradient_matches_central_differences_fp64(case):
    e0, grad, gom = energy_and_grads(case, case["c"], OMEGA, _lib.PREC_FP64)
    mir = synth.mirror_index(case["mill"])
    rng = np.random.default_rng(8)
    h = 1e-5
    for _ in range(8):
        d = rng.standard_normal(case["c"].shape) + 1j * rng.standard_normal(case["c"].shape)
        d = 0.5 * (d + np.conj(d[:, mir]))
        # scale the direction to the orbitals' norm: h d then changes c by ~1e-5
        # relative, which keeps the O(h^2) truncation of the quartic E_x far below 1e-6
        d *= np.linalg.norm(case["c"]) / np.linalg.norm(d)
        ep, _, _ = energy_and_grads(case, case["c"] + h * d, OMEGA, _lib.PREC_FP64)
        em, _, _ = energy_and_grads(case, case["c"] - h * d, OMEGA, _lib.PREC_FP64)
        slope = float(np.sum(np.conj(d) * grad).real)  # torch grad = 2 dE/dc*
        assert abs((ep - em) / (2 * h) - slope) <= 1e-6 * abs(slope)
    ep, _, _ = energy_and_grads(case, case["c"], OMEGA + h, _lib.PREC_FP64)
    em, _, _ = energy_and_grads(case, case["c"], OMEGA - h, _lib.PREC_FP64)
    assert abs((ep - em) / (2 * h) - gom) <= 1e-6 * abs(gom)


def test_mixed_gradient_matches_fp64_within_bound(case):
    e64, g64, o64 = energy_and_grads(case, case["c"], OMEGA, _lib.PREC_FP64)
    e32, g32, o32 = energy_and_grads(case, case["c"], OMEGA, _lib.PREC_MIXED32)
    assert abs(e32 - e64) <= 5e-6 * abs(e64)
    assert abs(o32 - o64) <= 5e-6 * abs(o64)
    assert rel_inf(g32, g64) <= 2e-5


def test_gradient_matches_the_oracle_on_eight_bands(case):
    c8 = np.ascontiguousarray(case["c"][:8])
    occ8 = np.array([2.0, 2.0, 2.0, 1.5, 1.0, 1.0, 0.5, 0.25])
    vref, eref, dref = oracle.fock_apply(c8, occ8, case["mill"], (N, N, N), case["cell"], "erfc", OMEGA)
    gref = 2.0 * occ8[:, None] * vref
    for prec, tol_g, tol_e in [(_lib.PREC_FP64, 1e-10, 1e-10), (_lib.PREC_MIXED32, 2e-5, 5e-6)]:
        e, g, gom = energy_and_grads(case, c8, OMEGA, prec, occ=occ8)
        assert rel_inf(g, gref) <= tol_g
        assert abs(e - eref) <= tol_e * abs(eref)
        assert abs(gom - dref) <= tol_e * abs(dref)


def test_complex64_orbitals_get_complex64_gradients(case):
    torch = case["torch"]
    psi = torch.from_numpy(case["c"][:4].astype(np.complex64)).cuda().requires_grad_(True)
    e = exchange_energy(psi, np.full(4, 2.0), N, case["cell"], ECUT, _lib.ERFC, OMEGA, _lib.PREC_MIXED32)
    e.backward()
    assert psi.grad.dtype == torch.complex64 and psi.grad.shape == psi.shape
