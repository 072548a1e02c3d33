"""The oracle against closed forms that plane-wave orbitals give (CPU).

A plane wave psi_G(r) = Omega^-1/2 exp(i G.r) times another has a single
Fourier component: psi_G'* psi_G = exp(i (G - G').r) / Omega.  The pair
potential is then v(G - G') times it, so when every orbital is a plane wave
each one is an eigenfunction of V_x (§4, V_x equation):

  V_x psi_G = lambda_G psi_G,   lambda_G = -(1/Omega) sum_G' f_G' v(G - G'),
  E_x = (1/2) sum_G f_G lambda_G = -(1/(2 Omega)) sum_{G,G'} f_G f_G' v(G - G'),

the exchange eigenvalue of plane-wave states (the electron-gas form, here with
the truncated or the screened kernel, both finite at G = G').  With Bloch
states exp(i (k + G).r) the kernel's argument is the momentum difference
(k + G) - (k' + G').  Orbitals that are a few plane waves each (sqrt(2)
cos(G.r), sqrt(2) sin(G.r)) follow from the same single-component products,
summed by hand below: pair by pair, rhot_ij(Q) = (1/Omega) sum over G' - G = Q
of c_i(G)* c_j(G'), the potential v(Q) rhot_ij(Q), and its product with psi_i
collected by frequency.  The grids are chosen so that no frequency of a
product wraps around (every Miller component stays below N/2), so the oracle's
grid transforms must reproduce these sums to rounding.

The kernels are evaluated here from their textbook transforms, in forms the
oracle does not use: the Spencer-Alavi kernel as 4 pi (1 - cos(G Rc)) / G^2
(the oracle writes 8 pi sin^2(G Rc / 2) / G^2), the erfc kernel with
1 - exp(...) (the oracle uses expm1); the kernels themselves are pinned by
radial quadrature in test_oracle_pins.py.
"""

import numpy as np
import pytest

import oracle
from oracle.kernels import ERFC, SPENCER_ALAVI
from oracle.lattice import cell_volume, gsphere_k, reciprocal_lattice

GENERAL_CELL = np.array([[7.0, 0.0, 0.0], [1.1, 7.6, 0.0], [0.4, -0.7, 8.3]])


def kernel(kind, q2, vol, omega):
    """v(Q) and dv/domega at |Q|^2 = q2 (scalars)."""
    if kind == SPENCER_ALAVI:
        rc = (3.0 * vol / (4.0 * np.pi)) ** (1.0 / 3.0)
        if q2 == 0.0:
            return 2.0 * np.pi * rc * rc, 0.0
        q = np.sqrt(q2)
        return 4.0 * np.pi * (1.0 - np.cos(q * rc)) / q2, 0.0
    e = np.exp(-q2 / (4.0 * omega * omega))
    dv = -(2.0 * np.pi / omega**3) * e
    if q2 == 0.0:
        return np.pi / (omega * omega), dv
    return 4.0 * np.pi * (1.0 - e) / q2, dv


def sphere_row(miller, m):
    hit = np.nonzero(np.all(miller == np.asarray(m), axis=1))[0]
    assert len(hit) == 1, "Miller index %r is not on the sphere" % (m,)
    return int(hit[0])


CASES = [(SPENCER_ALAVI, None), (ERFC, 0.37)]


@pytest.mark.parametrize("kind,omega", CASES, ids=["spencer_alavi", "erfc"])
def test_plane_waves_are_eigenfunctions_with_the_exchange_eigenvalue(kind, omega):
    # complex Gamma-point orbitals, one plane wave each, uneven occupations
    grid = (16, 16, 16)
    cell = GENERAL_CELL
    vol = cell_volume(cell)
    b = reciprocal_lattice(cell)
    miller, _ = oracle.gsphere(grid, cell, 4.0)
    waves = [(0, 0, 0), (1, 0, 0), (0, -1, 1), (-1, 1, 0), (1, 1, -1), (0, 0, -1)]
    occ = np.array([2.0, 1.5, 1.0, 0.5, 0.25, 2.0])
    c = np.zeros((len(waves), len(miller)), dtype=np.complex128)
    for n, m in enumerate(waves):
        c[n, sphere_row(miller, m)] = 1.0
    vpsi, ex, dex = oracle.fock_apply(c, occ, miller, grid, cell, kind, omega, real=False)

    gv = np.array(waves, dtype=np.float64) @ b
    lam = np.zeros(len(waves))
    dlam = np.zeros(len(waves))
    for j in range(len(waves)):
        for i in range(len(waves)):
            d = gv[j] - gv[i]
            v, dv = kernel(kind, float(d @ d), vol, omega)
            lam[j] -= occ[i] * v / vol
            dlam[j] -= occ[i] * dv / vol
    expect = lam[:, None] * c
    scale = np.max(np.abs(lam))
    assert np.max(np.abs(vpsi - expect)) <= 1e-12 * scale
    assert abs(ex - 0.5 * np.dot(occ, lam)) <= 1e-12 * abs(ex)
    assert abs(dex - 0.5 * np.dot(occ, dlam)) <= 1e-12 * max(abs(dex), 1e-300)


def sparse_exchange(orbs, occ, gvec_of, vol, kind, omega):
    """V_x psi_j and E_x of orbitals given as {Miller tuple: coefficient}, by
    single-component products collected per frequency (no grid)."""
    nb = len(orbs)
    out = [dict() for _ in range(nb)]
    ex = 0.0
    dex = 0.0
    for j in range(nb):
        for i in range(nb):
            rhot = {}
            for g, ci in orbs[i].items():
                for g2, cj in orbs[j].items():
                    q = tuple(a - b for a, b in zip(g2, g))
                    rhot[q] = rhot.get(q, 0.0) + np.conj(ci) * cj / vol
            for q, r in rhot.items():
                qv = gvec_of(q)
                v, dv = kernel(kind, float(qv @ qv), vol, omega)
                ex += -0.5 * vol * occ[i] * occ[j] * v * abs(r) ** 2
                dex += -0.5 * vol * occ[i] * occ[j] * dv * abs(r) ** 2
                for g, ci in orbs[i].items():
                    k = tuple(a + b for a, b in zip(g, q))
                    out[j][k] = out[j].get(k, 0.0) - occ[i] * ci * v * r
    return out, ex, dex


@pytest.mark.parametrize("kind,omega", CASES, ids=["spencer_alavi", "erfc"])
def test_real_cosine_and_sine_orbitals_match_the_sparse_fourier_sums(kind, omega):
    # real Gamma-point orbitals (c(-G) = c(G)*), the oracle's real path: a
    # constant, cosines and sines of a few reciprocal vectors
    grid = (16, 16, 16)
    cell = GENERAL_CELL
    vol = cell_volume(cell)
    b = reciprocal_lattice(cell)
    miller, _ = oracle.gsphere(grid, cell, 2.5)
    s = 1.0 / np.sqrt(2.0)
    orbs = [
        {(0, 0, 0): 1.0},
        {(1, 0, 0): s, (-1, 0, 0): s},                 # sqrt(2) cos(G.r)
        {(0, 1, -1): -1j * s, (0, -1, 1): 1j * s},     # sqrt(2) sin(G.r)
        {(1, 1, 0): 0.6 * s, (-1, -1, 0): 0.6 * s, (0, 0, 1): -0.8j * s, (0, 0, -1): 0.8j * s},
    ]
    occ = np.array([2.0, 1.0, 0.5, 1.5])
    c = np.zeros((len(orbs), len(miller)), dtype=np.complex128)
    for n, o in enumerate(orbs):
        for m, v in o.items():
            c[n, sphere_row(miller, m)] = v
    vpsi, ex, dex = oracle.fock_apply(c, occ, miller, grid, cell, kind, omega, real=True)

    exp_v, exp_e, exp_d = sparse_exchange(orbs, occ, lambda m: np.array(m, dtype=np.float64) @ b, vol, kind,
                                          omega)
    on_sphere = {tuple(int(x) for x in m): r for r, m in enumerate(miller)}
    expect = np.zeros_like(vpsi)
    for j in range(len(orbs)):
        for k, val in exp_v[j].items():
            if k in on_sphere:  # V_x psi is projected onto the sphere
                expect[j, on_sphere[k]] += val
    scale = np.max(np.abs(expect))
    assert scale > 0.0
    assert np.max(np.abs(vpsi - expect)) <= 1e-12 * scale
    # the orbitals reach frequencies off the sphere too (products of three)
    assert any(k not in on_sphere for d in exp_v for k in d)
    assert abs(ex - exp_e) <= 1e-12 * abs(exp_e)
    assert abs(dex - exp_d) <= 1e-12 * max(abs(exp_d), 1e-300)


@pytest.mark.parametrize("kind,omega", CASES, ids=["spencer_alavi", "erfc"])
def test_bloch_plane_waves_take_the_momentum_difference(kind, omega):
    # k points: states exp(i (k + G).r); the kernel's argument between state
    # (k, G) and state (k', G') is (k + G) - (k' + G'), whose G part alone
    # would differ by k - k'
    grid = (16, 16, 16)
    cell = GENERAL_CELL
    vol = cell_volume(cell)
    b = reciprocal_lattice(cell)
    kfrac = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.0, 0.25, -0.5]])
    weights = np.array([0.5, 0.25, 0.25])
    waves = {0: [(0, 0, 0), (1, 0, 0), (0, -1, 1)],
             1: [(-1, 0, 0), (0, 1, 0), (1, 0, -1)],
             2: [(0, 0, 1), (0, -1, 0), (1, 1, 0)]}
    occ = np.array([[2.0, 1.0, 0.5], [1.5, 2.0, 1.0], [0.75, 0.25, 2.0]])
    c_list, mill_list = [], []
    for k in range(3):
        mk, _ = gsphere_k(grid, cell, 5.0, kfrac[k])
        ck = np.zeros((3, len(mk)), dtype=np.complex128)
        for n, m in enumerate(waves[k]):
            ck[n, sphere_row(mk, m)] = 1.0
        c_list.append(ck)
        mill_list.append(mk)
    vk, ex = oracle.fock_apply_kpoints(c_list, occ, mill_list, kfrac, weights, grid, cell, kind, omega)

    def momentum(k, m):
        return (kfrac[k] + np.array(m, dtype=np.float64)) @ b

    ex_expect = 0.0
    for k in range(3):
        lam = np.zeros(3)
        for n in range(3):
            p = momentum(k, waves[k][n])
            for kp in range(3):
                for m in range(3):
                    d = p - momentum(kp, waves[kp][m])
                    v, _ = kernel(kind, float(d @ d), vol, omega)
                    lam[n] -= weights[kp] * occ[kp, m] * v / vol
        expect = lam[:, None] * c_list[k]
        assert np.max(np.abs(vk[k] - expect)) <= 1e-12 * np.max(np.abs(lam))
        ex_expect += 0.5 * weights[k] * np.dot(occ[k], lam)
    assert abs(ex - ex_expect) <= 1e-12 * abs(ex_expect)


@pytest.mark.parametrize("kind,omega", CASES, ids=["spencer_alavi", "erfc"])
def test_fixed_operator_on_trial_plane_waves(kind, omega):
    # V_x fixed by plane-wave occupied states, applied to trial plane waves
    # that are not among them (complex orbitals): each trial wave is an
    # eigenfunction with -(1/Omega) sum_i f_i v(G_a - G_i)
    grid = (16, 16, 16)
    cell = GENERAL_CELL
    vol = cell_volume(cell)
    b = reciprocal_lattice(cell)
    miller, _ = oracle.gsphere(grid, cell, 4.0)
    occupied = [(0, 0, 0), (1, 0, 0), (0, 1, -1)]
    occ = np.array([2.0, 1.25, 0.5])
    trial = [(-1, 0, 0), (0, 0, 1), (1, -1, 1), (0, 0, 0)]
    c_occ = np.zeros((len(occupied), len(miller)), dtype=np.complex128)
    c_tr = np.zeros((len(trial), len(miller)), dtype=np.complex128)
    for n, m in enumerate(occupied):
        c_occ[n, sphere_row(miller, m)] = 1.0
    for n, m in enumerate(trial):
        c_tr[n, sphere_row(miller, m)] = 1.0
    out = oracle.fock_apply_to(c_occ, occ, c_tr, miller, grid, cell, kind, omega, real=False)
    go = np.array(occupied, dtype=np.float64) @ b
    gt = np.array(trial, dtype=np.float64) @ b
    lam = np.zeros(len(trial))
    for a in range(len(trial)):
        for i in range(len(occupied)):
            d = gt[a] - go[i]
            lam[a] -= occ[i] * kernel(kind, float(d @ d), vol, omega)[0] / vol
    assert np.max(np.abs(out - lam[:, None] * c_tr)) <= 1e-12 * np.max(np.abs(lam))
