"""Pins of the FP64 oracle against mathematics it does not share code with.

Each test fixes a property that a plausible mistake in the oracle (a dropped
term, a wrong sign, an index or a transposed operand) would break.
"""

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from oracle.kernels import SPENCER_ALAVI, ERFC
from paper_1305_7313_gb300 import synth
from tests import _dft


def cubic(L):
    return (L * np.eye(3)).ravel()


def small_case(grid=(8, 8, 8), L=6.0, ecut=4.0, nb=4, seed=11, cell=None):
    cell = cubic(L) if cell is None else np.asarray(cell, dtype=np.float64)
    mill, _ = oracle.gsphere(grid, cell, ecut)
    c = synth.orbitals(mill, cell, nb, seed)
    return cell, mill, c


# ---------------------------------------------------------------- the sphere

def brute_force_sphere(cell, ecut, mmax=20):
    b = _dft.recip(cell)
    r = np.arange(-mmax, mmax + 1)
    pts = []
    for m1 in r:
        for m2 in r:
            for m3 in r:
                g = m1 * b[0] + m2 * b[1] + m3 * b[2]
                if 0.5 * float(g @ g) <= ecut:
                    pts.append((m1, m2, m3))
    return pts


@pytest.mark.parametrize("L,ecut,npw", [(10.0, 10.0, 1503)])
def test_sphere_count_matches_brute_force(L, ecut, npw):
    cell = cubic(L)
    mill, g2 = oracle.gsphere((24, 24, 24), cell, ecut)
    assert len(mill) == npw == len(brute_force_sphere(cell, ecut, 9))
    assert set(map(tuple, mill.tolist())) == set(brute_force_sphere(cell, ecut, 9))


def test_sphere_counts_of_large_cells():
    # the sphere of a cubic cell is the set of integer m with |m|^2 <= 2 Ecut / b^2
    for L, ecut, npw in [(27.0, 12.0, 39127), (20.0, 12.0, 15895)]:
        bound = 2.0 * ecut / (2.0 * np.pi / L) ** 2
        r = np.arange(-30, 31)
        m2 = (r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2)
        assert int(np.sum(m2 <= bound)) == npw
        mill, _ = oracle.gsphere((96, 96, 96), cubic(L), ecut)
        assert len(mill) == npw


def test_sphere_order_and_symmetry_general_cell():
    cell = np.array([[7.0, 0.3, 0.0], [0.5, 8.0, 0.2], [0.0, -0.4, 6.5]])
    mill, g2 = oracle.gsphere((24, 24, 24), cell, 6.0)
    assert set(map(tuple, mill.tolist())) == set(brute_force_sphere(cell, 6.0, 10))
    # ascending |G|^2, ties lexicographic
    for k in range(len(mill) - 1):
        assert g2[k] < g2[k + 1] or (g2[k] == g2[k + 1] and tuple(mill[k]) < tuple(mill[k + 1]))
    assert tuple(mill[0]) == (0, 0, 0)
    s = set(map(tuple, mill.tolist()))
    assert all((-a, -b, -c) in s for a, b, c in s)


def test_sphere_too_big_for_grid_is_rejected():
    with pytest.raises(ValueError):
        oracle.gsphere((12, 12, 12), cubic(10.0), 10.0)


# --------------------------------------------------------------- the kernels

def test_spencer_alavi_is_the_truncated_coulomb_transform():
    vol = 1000.0
    rc = oracle.spencer_alavi_rc(vol)
    assert abs(rc - 6.2035049089940) < 1e-9
    for g in [0.3, 1.1, 2.7, 5.0]:
        # int_{|r|<Rc} exp(-iG.r)/r d^3r = (4 pi / G) int_0^Rc sin(G r) dr
        ref = 4.0 * np.pi / g * integrate.quad(lambda r: np.sin(g * r), 0.0, rc, limit=200)[0]
        assert abs(oracle.coulomb_kernel(SPENCER_ALAVI, np.array([g * g]), vol)[0] - ref) < 1e-9 * ref
    v0 = oracle.coulomb_kernel(SPENCER_ALAVI, np.array([0.0]), vol)[0]
    assert abs(v0 - 4.0 * np.pi * integrate.quad(lambda r: r, 0.0, rc)[0]) < 1e-9
    assert abs(oracle.coulomb_kernel(SPENCER_ALAVI, np.array([0.0]), 27.0**3)[0] - 1762.71) < 0.01


def test_erfc_kernel_is_the_screened_coulomb_transform():
    om = 0.106
    assert abs(oracle.coulomb_kernel(ERFC, np.array([0.0]), 1.0, om)[0] - 279.60) < 0.01
    for g in [0.05, 0.4, 1.3]:
        f = lambda r: special.erfc(om * r) * np.sin(g * r)
        ref = 4.0 * np.pi / g * integrate.quad(f, 0.0, 80.0 / om, limit=2000)[0]
        assert abs(oracle.coulomb_kernel(ERFC, np.array([g * g]), 1.0, om)[0] - ref) < 1e-7 * ref
    g2 = np.array([0.0, 0.01, 0.05, 0.5])
    h = 1e-6
    fd = (oracle.coulomb_kernel(ERFC, g2, 1.0, om + h) - oracle.coulomb_kernel(ERFC, g2, 1.0, om - h)) / (2 * h)
    assert np.allclose(oracle.coulomb_kernel_domega(ERFC, g2, 1.0, om), fd, rtol=1e-6, atol=0)


# ------------------------------------------------------ the chain, by DFT

@pytest.mark.parametrize("grid,L,ecut,nb,kind", [
    ((6, 6, 6), 5.0, 2.5, 3, SPENCER_ALAVI),
    ((8, 8, 8), 6.0, 4.0, 4, ERFC),
    ((12, 12, 12), 7.0, 6.0, 3, SPENCER_ALAVI),
])
def test_oracle_matches_direct_dft(grid, L, ecut, nb, kind):
    cell, mill, c = small_case(grid, L, ecut, nb, seed=3)
    occ = np.linspace(2.0, 1.0, nb)
    omega = 0.7 if kind == ERFC else None
    vol = L ** 3
    vpsi, ex, _ = oracle.fock_apply(c, occ, mill, grid, cell, kind, omega)
    vref, eref = _dft.fock_direct(c, occ, mill, grid, cell,
                                  lambda g2: oracle.coulomb_kernel(kind, g2, vol, omega))
    assert abs(ex - eref) <= 1e-12 * abs(eref)
    assert np.max(np.abs(vpsi - vref)) <= 1e-12 * np.max(np.abs(vref))


def test_oracle_matches_direct_dft_general_cell_complex_orbitals():
    grid = (8, 8, 8)
    cell = np.array([[6.0, 0.4, 0.0], [0.0, 6.5, 0.3], [0.2, 0.0, 5.5]])
    mill, _ = oracle.gsphere(grid, cell, 3.0)
    rng = np.random.default_rng(5)
    c = rng.standard_normal((3, len(mill))) + 1j * rng.standard_normal((3, len(mill)))
    occ = np.array([2.0, 1.5, 0.5])
    vol = abs(np.linalg.det(cell.reshape(3, 3)))
    vpsi, ex, _ = oracle.fock_apply(c, occ, mill, grid, cell, SPENCER_ALAVI, real=False)
    vref, eref = _dft.fock_direct(c, occ, mill, grid, cell,
                                  lambda g2: oracle.coulomb_kernel(SPENCER_ALAVI, g2, vol))
    assert abs(ex - eref) <= 1e-12 * abs(eref)
    assert np.max(np.abs(vpsi - vref)) <= 1e-12 * np.max(np.abs(vref))


# ------------------------------------------------ closed-form self-energies

@pytest.mark.parametrize("kind,omega", [(SPENCER_ALAVI, None), (ERFC, 0.5)])
def test_gaussian_self_exchange(kind, omega):
    sigma, L, n, ecut = 1.0, 30.0, 96, 16.0
    cell = cubic(L)
    mill, _ = oracle.gsphere((n, n, n), cell, ecut)
    c = synth.gaussian_orbital(mill, cell, sigma)
    _, ex, _ = oracle.fock_apply(c, np.array([1.0]), mill, (n, n, n), cell, kind, omega)
    expect = -1.0 / (2.0 * np.sqrt(np.pi) * sigma)
    if kind == ERFC:
        expect += 1.0 / np.sqrt(2.0 * np.pi * (2.0 * sigma**2 + 1.0 / (2.0 * omega**2)))
    assert abs(ex - expect) < 1e-10


# ------------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def cfg_small():
    grid = (24, 24, 24)
    cell = cubic(10.0)
    mill, _ = oracle.gsphere(grid, cell, 10.0)
    c = synth.orbitals(mill, cell, 8, 1305)
    occ = np.full(8, 2.0)
    vpsi, ex, _ = oracle.fock_apply(c, occ, mill, grid, cell, SPENCER_ALAVI)
    return dict(grid=grid, cell=cell, mill=mill, c=c, occ=occ, vpsi=vpsi, ex=ex)


def test_vx_is_hermitian_and_negative_semidefinite(cfg_small):
    m = oracle.overlap_matrix_vx(cfg_small["c"], cfg_small["vpsi"])
    assert np.max(np.abs(m - m.conj().T)) <= 1e-13 * np.max(np.abs(m))
    ev = np.linalg.eigvalsh(0.5 * (m + m.conj().T))
    assert ev.max() <= 1e-12 * np.max(np.abs(m))
    assert ev.min() < 0.0


def test_energy_identity(cfg_small):
    e2 = oracle.exchange_energy_from_vpsi(cfg_small["c"], cfg_small["occ"], cfg_small["vpsi"])
    assert abs(e2 - cfg_small["ex"]) <= 1e-12 * abs(cfg_small["ex"])
    assert cfg_small["ex"] < 0.0


def test_real_orbitals_give_hermitian_coefficients(cfg_small):
    mir = synth.mirror_index(cfg_small["mill"])
    v = cfg_small["vpsi"]
    assert np.max(np.abs(v[:, mir] - np.conj(v))) <= 1e-13 * np.max(np.abs(v))


def test_unitary_invariance(cfg_small):
    rng = np.random.default_rng(7)
    q, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    c2 = q.T @ cfg_small["c"]
    v2, e2, _ = oracle.fock_apply(c2, cfg_small["occ"], cfg_small["mill"], cfg_small["grid"],
                                  cfg_small["cell"], SPENCER_ALAVI)
    assert abs(e2 - cfg_small["ex"]) <= 1e-12 * abs(cfg_small["ex"])
    assert np.max(np.abs(v2 - q.T @ cfg_small["vpsi"])) <= 1e-12 * np.max(np.abs(v2))


def test_translation_by_grid_vector(cfg_small):
    # psi'(r) = psi(r - t) with t = (3/24) a1 + (5/24) a2: c'(G) = c(G) exp(-i G.t)
    m = cfg_small["mill"].astype(np.float64)
    ph = np.exp(-2j * np.pi * (m[:, 0] * 3 / 24 + m[:, 1] * 5 / 24))
    c2 = cfg_small["c"] * ph[None, :]
    v2, e2, _ = oracle.fock_apply(c2, cfg_small["occ"], cfg_small["mill"], cfg_small["grid"],
                                  cfg_small["cell"], SPENCER_ALAVI)
    assert abs(e2 - cfg_small["ex"]) <= 1e-12 * abs(cfg_small["ex"])
    assert np.max(np.abs(v2 - cfg_small["vpsi"] * ph[None, :])) <= 1e-12 * np.max(np.abs(v2))


def test_permutation_and_partition_invariance(cfg_small):
    perm = np.array([3, 0, 7, 5, 1, 2, 6, 4])
    v2, e2, _ = oracle.fock_apply(cfg_small["c"][perm], cfg_small["occ"], cfg_small["mill"],
                                  cfg_small["grid"], cfg_small["cell"], SPENCER_ALAVI)
    assert abs(e2 - cfg_small["ex"]) <= 1e-12 * abs(cfg_small["ex"])
    assert np.max(np.abs(v2 - cfg_small["vpsi"][perm])) <= 1e-12 * np.max(np.abs(v2))
    parts = [[0, 5], [1, 2, 7], [3], [4, 6]]
    vs, es = 0.0, 0.0
    for p in parts:
        v, e, _ = oracle.fock_apply(cfg_small["c"], cfg_small["occ"], cfg_small["mill"],
                                    cfg_small["grid"], cfg_small["cell"], SPENCER_ALAVI, src_bands=p)
        vs = vs + v
        es += e
    assert abs(es - cfg_small["ex"]) <= 1e-12 * abs(cfg_small["ex"])
    assert np.max(np.abs(vs - cfg_small["vpsi"])) <= 1e-12 * np.max(np.abs(vs))


def test_occupations_enter_linearly_per_band():
    # doubling every f_i scales V_x psi by 2 and E_x by 4
    cell, mill, c = small_case()
    occ = np.array([2.0, 1.0, 0.5, 1.5])
    v1, e1, _ = oracle.fock_apply(c, occ, mill, (8, 8, 8), cell, SPENCER_ALAVI)
    v2, e2, _ = oracle.fock_apply(c, 2 * occ, mill, (8, 8, 8), cell, SPENCER_ALAVI)
    assert np.allclose(v2, 2 * v1, rtol=1e-13, atol=0)
    assert abs(e2 - 4 * e1) <= 1e-13 * abs(e2)


# -------------------------------------------------------- gradients by FD

def test_gradient_matches_central_differences():
    grid = (12, 12, 12)
    cell, mill, c = small_case(grid, 7.0, 6.0, 4, seed=9)
    occ = np.array([2.0, 2.0, 1.0, 0.5])
    vpsi, _, _ = oracle.fock_apply(c, occ, mill, grid, cell, ERFC, 0.4)
    mir = synth.mirror_index(mill)
    rng = np.random.default_rng(13)
    h = 1e-5
    for _ in range(3):
        d = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)
        d = 0.5 * (d + np.conj(d[:, mir]))              # keeps psi real
        ep = oracle.fock_apply(c + h * d, occ, mill, grid, cell, ERFC, 0.4)[1]
        em = oracle.fock_apply(c - h * d, occ, mill, grid, cell, ERFC, 0.4)[1]
        slope = 2.0 * np.sum(occ[:, None] * (vpsi * np.conj(d))).real
        assert abs((ep - em) / (2 * h) - slope) <= 1e-7 * abs(slope)


def test_omega_derivative_matches_central_differences():
    grid = (12, 12, 12)
    cell, mill, c = small_case(grid, 7.0, 6.0, 3, seed=4)
    occ = np.full(3, 2.0)
    _, _, dex = oracle.fock_apply(c, occ, mill, grid, cell, ERFC, 0.3)
    h = 1e-5
    ep = oracle.fock_apply(c, occ, mill, grid, cell, ERFC, 0.3 + h)[1]
    em = oracle.fock_apply(c, occ, mill, grid, cell, ERFC, 0.3 - h)[1]
    assert abs((ep - em) / (2 * h) - dex) <= 1e-7 * abs(dex)


# ------------------------------------------- V_x applied to trial orbitals

def test_fixed_operator_on_trial_orbitals_matches_direct_dft():
    grid = (8, 8, 8)
    cell, mill, c = small_case(grid, 6.0, 4.0, 5, seed=21)
    occ = np.array([2.0, 1.5, 1.0, 0.5, 0.25])
    trial = synth.orbitals(mill, cell, 3, 77)
    v = oracle.fock_apply_to(c, occ, trial, mill, grid, cell, ERFC, 0.6)
    vref = _dft.fock_direct_to(c, occ, trial, mill, grid, cell,
                               lambda g2: oracle.coulomb_kernel(ERFC, g2, 6.0 ** 3, 0.6))
    assert np.max(np.abs(v - vref)) <= 1e-12 * np.max(np.abs(vref))


def test_fixed_operator_on_the_occupied_set_is_the_fock_apply(cfg_small):
    v = oracle.fock_apply_to(cfg_small["c"], cfg_small["occ"], cfg_small["c"], cfg_small["mill"],
                             cfg_small["grid"], cfg_small["cell"], SPENCER_ALAVI)
    assert np.max(np.abs(v - cfg_small["vpsi"])) <= 1e-13 * np.max(np.abs(v))


def test_fixed_operator_is_linear_and_hermitian_on_trial_functions():
    grid = (12, 12, 12)
    cell, mill, c = small_case(grid, 7.0, 6.0, 4, seed=5)
    occ = np.full(4, 2.0)
    t = synth.orbitals(mill, cell, 3, 6)
    v = oracle.fock_apply_to(c, occ, t, mill, grid, cell, SPENCER_ALAVI)
    m = np.conj(t) @ v.T
    assert np.max(np.abs(m - m.conj().T)) <= 1e-13 * np.max(np.abs(m))
    comb = 0.3 * t[0] - 1.7 * t[2]
    vc = oracle.fock_apply_to(c, occ, comb[None, :], mill, grid, cell, SPENCER_ALAVI)[0]
    assert np.max(np.abs(vc - (0.3 * v[0] - 1.7 * v[2]))) <= 1e-13 * np.max(np.abs(vc))
