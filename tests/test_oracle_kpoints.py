"""Pins of the k-point oracle: the Gamma limit, an exact supercell identity
(Brillouin-zone sampling of a cell equals the Gamma point of the supercell
that unfolds it), Hermiticity within each k, and the E_x identity."""

import numpy as np

import oracle
from oracle.kernels import ERFC, SPENCER_ALAVI
from paper_1305_7313_gb300 import synth


def test_single_gamma_point_is_the_gamma_oracle_with_complex_orbitals():
    # 8^3 at L = 6, Ecut = 4: the pair densities alias (|m| reaches 8 > 4), and
    # the k-point sum at k = 0 is still the Gamma sum term by term
    grid = (8, 8, 8)
    cell = (6.0 * np.eye(3)).ravel()
    mill, _ = oracle.gsphere(grid, cell, 4.0)
    mk, _ = oracle.gsphere_k(grid, cell, 4.0, (0.0, 0.0, 0.0))
    assert np.array_equal(mill, mk)
    c = synth.orbitals_k(mk, cell, (0, 0, 0), 4, 3)
    occ = np.array([2.0, 1.5, 1.0, 0.5])
    v1, e1, _ = oracle.fock_apply(c, occ, mill, grid, cell, ERFC, 0.5, real=False)
    vk, ek = oracle.fock_apply_kpoints([c], occ[None, :], [mk], [[0, 0, 0]], [1.0], grid, cell, ERFC, 0.5)
    assert abs(ek - e1) <= 1e-13 * abs(e1)
    assert np.max(np.abs(vk[0] - v1)) <= 1e-13 * np.max(np.abs(v1))


def test_two_k_points_equal_the_gamma_point_of_the_doubled_cell():
    # cell (L1, L, L) sampled at k = 0 and k = b1/2 (weights 1/2) is the Gamma
    # point of the supercell (2 L1, L, L): k + G = 2 (m1 + kf1) b1' + m2 b2 + m3 b3
    # on grids that alias the pair densities: the identity is exact for the
    # plain sum over ordered pairs on any pair of matching grids
    L1, L, ecut, nb = 5.0, 6.0, 3.0, 3
    grid, sgrid = (8, 8, 8), (16, 8, 8)
    cell = np.diag([L1, L, L]).ravel()
    scell = np.diag([2 * L1, L, L]).ravel()
    kf = np.array([[0.0, 0, 0], [0.5, 0, 0]])
    mills, cs = [], []
    for k in range(2):
        m, _ = oracle.gsphere_k(grid, cell, ecut, kf[k])
        mills.append(m)
        cs.append(synth.orbitals_k(m, cell, kf[k], nb, 10 + k))
    occ = np.array([[2.0, 1.0, 0.5], [1.5, 1.0, 0.25]])
    vk, ek = oracle.fock_apply_kpoints(cs, occ, mills, kf, [0.5, 0.5], grid, cell, ERFC, 0.45)
    # unfold
    smill, _ = oracle.gsphere(sgrid, scell, ecut)
    index = {tuple(r): i for i, r in enumerate(smill.tolist())}
    cs_super = np.zeros((2 * nb, len(smill)), dtype=np.complex128)
    maps = []
    for k in range(2):
        sm = mills[k].copy()
        sm[:, 0] = 2 * sm[:, 0] + int(round(2 * kf[k, 0]))
        idx = np.array([index[tuple(r)] for r in sm.tolist()])
        maps.append(idx)
        cs_super[k * nb:(k + 1) * nb, idx] = cs[k]
    assert sum(len(m) for m in mills) == len(smill)
    vs, es, _ = oracle.fock_apply(cs_super, occ.ravel(), smill, sgrid, scell, ERFC, 0.45, real=False)
    assert abs(es - 2.0 * ek) <= 1e-12 * abs(es)
    for k in range(2):
        assert np.max(np.abs(vs[k * nb:(k + 1) * nb][:, maps[k]] - vk[k])) <= 1e-12 * np.max(np.abs(vk[k]))


def test_kpoint_operator_is_hermitian_per_k_and_gives_the_energy():
    grid = (12, 12, 12)
    cell = (7.0 * np.eye(3)).ravel()
    kf = np.array([[0.0, 0, 0], [0.5, 0, 0], [0.0, 0.5, 0.5], [0.25, -0.25, 0.5]])
    w = np.array([0.4, 0.2, 0.3, 0.1])
    mills, cs = [], []
    for k in range(4):
        m, _ = oracle.gsphere_k(grid, cell, 5.0, kf[k])
        mills.append(m)
        cs.append(synth.orbitals_k(m, cell, kf[k], 3, 30 + k))
    occ = np.full((4, 3), 2.0)
    vk, ek = oracle.fock_apply_kpoints(cs, occ, mills, kf, w, grid, cell, SPENCER_ALAVI)
    e2 = 0.0
    for k in range(4):
        m = np.conj(cs[k]) @ vk[k].T
        assert np.max(np.abs(m - m.conj().T)) <= 1e-12 * np.max(np.abs(m))
        assert np.linalg.eigvalsh(0.5 * (m + m.conj().T)).max() <= 1e-12 * np.max(np.abs(m))
        e2 += 0.5 * w[k] * float(np.sum(occ[k] * np.diag(m).real))
    assert abs(e2 - ek) <= 1e-12 * abs(ek)


def test_kpoint_operator_is_hermitian_per_k_on_an_aliasing_grid():
    # the pair densities reach the Nyquist planes (|m| up to 8 on 8^3); within
    # one k, <psi_a|V_x|psi_b> = -sum over k', m of sum_G conj(rho_ma) v(G + q) rho_mb
    # with the same real kernel for a and b, so the matrix stays Hermitian
    grid = (8, 8, 8)
    cell = (6.0 * np.eye(3)).ravel()
    kf = np.array([[0.0, 0, 0], [0.5, 0.25, 0]])
    mills, cs = [], []
    for k in range(2):
        m, _ = oracle.gsphere_k(grid, cell, 4.0, kf[k])
        mills.append(m)
        cs.append(synth.orbitals_k(m, cell, kf[k], 3, 70 + k))
    vk, ek = oracle.fock_apply_kpoints(cs, np.full((2, 3), 2.0), mills, kf, [0.5, 0.5], grid, cell, ERFC, 0.7)
    e2 = 0.0
    for k in range(2):
        m = np.conj(cs[k]) @ vk[k].T
        assert np.max(np.abs(m - m.conj().T)) <= 1e-13 * np.max(np.abs(m))
        e2 += 0.5 * 0.5 * float(np.sum(2.0 * np.diag(m).real))
    assert abs(e2 - ek) <= 1e-12 * abs(ek)
