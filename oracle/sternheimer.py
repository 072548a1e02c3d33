"""Sternheimer linear response by conjugate gradients with converged /
unconverged band regrouping (oracle; test infrastructure).

The paper's §3.1 ("The Sternheimer equation") replaces the Green's-function
application of GIPAW by the linear systems

    (H - eps_n + alpha P) |g_n> = -Q |w_n>,      n = 0 .. nrhs-1,

with P = sum over occupied states of |u_i><u_i| (the projector on the occupied
manifold, here at one k point: k + q = k), Q = 1 - P, and alpha twice the
bandwidth of the occupied states so that the left-hand side is positive
definite.  They are solved by CG.  The paper's bookkeeping: the first CG
iteration updates every band; from the second on, the bands are split into
two groups, each contiguous in memory (not yet converged, converged), and only
the first group is updated; a band is converged when its residual norm falls
below a threshold; before returning, the bands are put back in their original
order.

Readings (the paper gives no H of its own here; GIPAW's is the Kohn-Sham
Hamiltonian):

* H is a model Kohn-Sham Hamiltonian on the plane-wave sphere S at the Gamma
  point: H = -1/2 nabla^2 + V(r), i.e. (H c)(G) = |G|^2/2 c(G) +
  (sqrt(Omega)/Ntot) FFT[V(r) psi(r)](G) for G in S, psi(r) = Omega^-1/2
  sum_G c(G) exp(iG.r) on the FFT grid, V a real local potential on the grid.
* Kets are Gamma-point real functions (c(-G) = c(G)*), so every inner
  product <a|b> = sum_G conj(a(G)) b(G) is real.
* The residual of band n is r_n = b_n - A_n g_n, b_n = -Q w_n, A_n = H - eps_n
  + alpha P; band n is converged when ||r_n|| < tol.  The starting guess is
  g_n = 0.  Plain CG, no preconditioner.
"""

import numpy as np

from .fock import orbitals_to_real, real_to_sphere
from .lattice import g2_of_miller, reciprocal_lattice


def kinetic(miller, cell):
    """|G|^2 / 2 on the sphere."""
    return 0.5 * g2_of_miller(miller, reciprocal_lattice(cell))


def apply_h(c, vloc, miller, grid, cell):
    """H c for kets c [m, npw]: kinetic term on the sphere plus the local
    potential applied in real space (the FFT route of §3-4)."""
    c = np.atleast_2d(np.asarray(c, dtype=np.complex128))
    psi = orbitals_to_real(c, miller, grid, cell, real=True)
    vpsi = real_to_sphere(np.asarray(vloc)[None] * psi, miller, grid, cell)
    return kinetic(miller, cell)[None, :] * c + np.atleast_2d(vpsi)


def apply_p(c, u):
    """P c = sum_i u_i <u_i|c> for kets c [m, npw] and occupied states u [nocc, npw]."""
    return (np.conj(u) @ np.atleast_2d(c).T).real.T @ u


def sternheimer_solve(u, eps, w, vloc, miller, grid, cell, alpha, tol, maxiter=1000):
    """g [nrhs, npw] solving (H - eps_n + alpha P) g_n = -Q w_n, by CG with the
    paper's regrouping of converged and unconverged bands.

    Returns ``(g, iterations [nrhs], residual norms [nrhs])``; iterations[n]
    counts the CG updates band n received.
    """
    u = np.atleast_2d(np.asarray(u, dtype=np.complex128))
    w = np.atleast_2d(np.asarray(w, dtype=np.complex128))
    eps = np.asarray(eps, dtype=np.float64)
    nrhs = w.shape[0]

    def apply_a(c, e):
        return apply_h(c, vloc, miller, grid, cell) - e[:, None] * c + alpha * apply_p(c, u)

    # working arrays in the order "position" (regrouped); order[k] = band at position k
    order = np.arange(nrhs)
    b = -(w - apply_p(w, u))
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.einsum("ng,ng->n", np.conj(r), r).real
    iters = np.zeros(nrhs, dtype=np.int64)
    m = nrhs  # positions [0, m) are not converged
    for it in range(maxiter):
        if m == 0:
            break
        e = eps[order[:m]]
        ap = apply_a(p[:m], e)
        pap = np.einsum("ng,ng->n", np.conj(p[:m]), ap).real
        a = rr[:m] / pap
        x[:m] += a[:, None] * p[:m]
        r[:m] -= a[:, None] * ap
        rr_new = np.einsum("ng,ng->n", np.conj(r[:m]), r[:m]).real
        iters[order[:m]] += 1
        beta = rr_new / rr[:m]
        rr[:m] = rr_new
        p[:m] = r[:m] + beta[:, None] * p[:m]
        # regroup: not converged first, converged after, both in their order
        done = np.sqrt(rr_new) < tol
        keep = np.concatenate([np.flatnonzero(~done), np.flatnonzero(done), np.arange(m, nrhs)])
        order, x, r, p, rr = order[keep], x[keep], r[keep], p[keep], rr[keep]
        m = int(np.count_nonzero(~done))
    # back to the original band order
    inv = np.argsort(order)
    return x[inv], iters, np.sqrt(rr[inv])


def dense_operator(vloc, miller, grid, cell):
    """The matrix of H on the sphere: H_GG' = |G|^2/2 delta_GG' + Vt(G - G'), with
    Vt(m) = FFT(V)(m) / Ntot at the grid index of m (indices modulo the grid),
    the exact matrix of the FFT route of apply_h."""
    grid = tuple(int(n) for n in grid)
    ntot = grid[0] * grid[1] * grid[2]
    vt = np.fft.fftn(np.asarray(vloc, dtype=np.complex128)) / ntot
    m = np.asarray(miller, dtype=np.int64)
    d = m[:, None, :] - m[None, :, :]
    h = vt[d[..., 0] % grid[0], d[..., 1] % grid[1], d[..., 2] % grid[2]]
    return h + np.diag(kinetic(miller, cell))
