"""Pins of the Sternheimer oracle (§3.1): the FFT route of the model H against
the dense matrix built from the potential's Fourier coefficients, that matrix
against closed forms, and the CG solution with band regrouping against a
direct dense solve of the same linear systems."""

import numpy as np

import oracle
from oracle.sternheimer import apply_h, apply_p, dense_operator, kinetic, sternheimer_solve
from paper_1305_7313_gb300 import synth

GRID = (12, 12, 12)
L, ECUT = 6.0, 4.0


def _cell():
    return (L * np.eye(3)).ravel()


def model_potential(grid, cell, seed=7, depth=1.5, width=0.9, centers=3):
    """The seeded model potential of the input generator (Gaussian wells)."""
    return synth.model_potential(grid, cell, seed, depth, width, centers)


def occupied_states(h, mill, nocc):
    """The nocc lowest eigenpairs of the dense H, each eigenvector turned into
    a Gamma-point real ket (c(-G) = c(G)*) by its phase."""
    e, v = np.linalg.eigh(h)
    mir = synth.mirror_index(mill)
    out = []
    for k in range(nocc):
        c = v[:, k]
        g = int(np.argmax(np.abs(c)))
        phase = c[mir[g]] / np.conj(c[g])  # c(-G) = phase c(G)*
        c = c * np.sqrt(np.conj(phase))
        assert np.max(np.abs(c[mir] - np.conj(c))) < 1e-10
        out.append(c)
    return e[:nocc], np.array(out)


def case(nocc=4, seed=7):
    cell = _cell()
    mill, _ = oracle.gsphere(GRID, cell, ECUT)
    v = model_potential(GRID, cell, seed)
    h = dense_operator(v, mill, GRID, cell)
    eps, u = occupied_states(h, mill, nocc)
    w = synth.orbitals(mill, cell, nocc, seed + 100)
    alpha = 2.0 * (eps[-1] - eps[0])
    return cell, mill, v, h, eps, u, w, alpha


def test_fft_route_equals_the_dense_matrix():
    cell, mill, v, h, eps, u, w, alpha = case()
    c = synth.orbitals(mill, cell, 5, 3)
    assert np.max(np.abs(apply_h(c, v, mill, GRID, cell) - c @ h.T)) <= 1e-13 * np.max(np.abs(h))
    assert np.max(np.abs(h - h.conj().T)) <= 1e-14 * np.max(np.abs(h))


def test_dense_matrix_closed_forms():
    cell = _cell()
    mill, _ = oracle.gsphere(GRID, cell, ECUT)
    # a constant potential shifts the kinetic diagonal
    h = dense_operator(np.full(GRID, -0.7), mill, GRID, cell)
    assert np.allclose(h, np.diag(kinetic(mill, cell) - 0.7), atol=1e-14)
    # V(r) = cos(b1 . r): Fourier coefficients 1/2 at m = +-(1, 0, 0)
    n1 = np.arange(GRID[0])[:, None, None] * np.ones(GRID)
    h = dense_operator(np.cos(2 * np.pi * n1 / GRID[0]), mill, GRID, cell)
    off = h - np.diag(np.diag(h))
    d = mill[:, None, :] - mill[None, :, :]
    unit = (np.abs(d[..., 0]) == 1) & (d[..., 1] == 0) & (d[..., 2] == 0)
    assert np.allclose(off[unit], 0.5, atol=1e-14) and np.allclose(off[~unit], 0.0, atol=1e-14)
    assert abs(kinetic(np.array([[1, 0, 0]]), cell)[0] - 0.5 * (2 * np.pi / L) ** 2) < 1e-14


def test_cg_with_regrouping_matches_a_direct_solve():
    cell, mill, v, h, eps, u, w, alpha = case()
    q_w = w - apply_p(w, u)
    g, iters, res = sternheimer_solve(u, eps, w, v, mill, GRID, cell, alpha, tol=1e-12)
    p = u.T @ np.conj(u)  # sum_i |u_i><u_i| as a matrix
    for n in range(len(eps)):
        a = h - eps[n] * np.eye(len(mill)) + alpha * p
        assert np.linalg.eigvalsh(a).min() > 0  # alpha = twice the occupied bandwidth
        g_direct = np.linalg.solve(a, -q_w[n])
        assert np.max(np.abs(g[n] - g_direct)) <= 1e-9 * np.max(np.abs(g_direct))
        assert res[n] < 1e-12
    assert np.max(np.abs(g[:, synth.mirror_index(mill)] - np.conj(g))) < 1e-12  # real kets


def test_regrouping_freezes_converged_bands_and_restores_the_order():
    # bands whose right-hand sides differ by orders of magnitude converge after
    # different numbers of updates; the frozen ones are not updated again, the
    # result is the direct solve, and a permuted input gives the permuted output
    cell, mill, v, h, eps, u, w, alpha = case()
    w = w * np.array([1.0, 1e-6, 1e-3, 1e-9])[:, None]
    g, iters, res = sternheimer_solve(u, eps, w, v, mill, GRID, cell, alpha, tol=1e-10)
    assert len(set(iters.tolist())) > 1 and iters[3] < iters[0]
    assert np.all(res < 1e-10)
    perm = np.array([2, 0, 3, 1])
    g2, iters2, _ = sternheimer_solve(u, eps[perm], w[perm], v, mill, GRID, cell, alpha, tol=1e-10)
    assert np.array_equal(iters2, iters[perm])
    assert np.max(np.abs(g2 - g[perm])) <= 1e-14 * np.max(np.abs(g))
