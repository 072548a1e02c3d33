"""Direct O(N^2) evaluation of the exchange chain on tiny grids.

An independent check of the oracle: plane-wave sums and DFT matrices written
out element by element, no FFT library.
"""

import numpy as np


def recip(cell):
    return 2.0 * np.pi * np.linalg.inv(np.asarray(cell, dtype=np.float64).reshape(3, 3)).T


def grid_points(grid):
    n = np.stack(np.meshgrid(*[np.arange(k) for k in grid], indexing="ij"), -1).reshape(-1, 3)
    return n


def grid_freqs(grid):
    """Miller index of each point in C order, fftfreq convention."""
    m = grid_points(grid).copy()
    for a, k in enumerate(grid):
        m[:, a] = np.where(m[:, a] < (k + 1) // 2, m[:, a], m[:, a] - k)
    return m


def phase(m, n, grid):
    """exp(2 pi i sum_a m_a n_a / N_a) for every (m, n) pair: shape (len(m), len(n))."""
    x = np.zeros((m.shape[0], n.shape[0]))
    for a, k in enumerate(grid):
        x += np.outer(m[:, a], n[:, a]) / float(k)
    return np.exp(2j * np.pi * x)


def fock_direct(c, occ, miller, grid, cell, vfun):
    """V_x psi (on the sphere) and E_x from direct sums. ``vfun(g2)`` gives v(G)."""
    a = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    vol = abs(np.linalg.det(a))
    pts = grid_points(grid)
    ntot = pts.shape[0]
    fr = grid_freqs(grid)
    b = recip(cell)
    g2 = np.einsum("gx,gx->g", fr @ b, fr @ b)
    v = vfun(g2)
    e_sphere = phase(np.asarray(miller), pts, grid)       # exp(+i G.r)   [npw, ntot]
    fwd = np.conj(phase(fr, pts, grid))                   # exp(-i G.r)   [ntot, ntot]
    psi = (c @ e_sphere) / np.sqrt(vol)                   # [nb, ntot]
    nb = c.shape[0]
    w = np.zeros_like(psi)
    ex = 0.0
    for j in range(nb):
        for i in range(nb):
            rho = np.conj(psi[i]) * psi[j]
            rhot = fwd @ rho / ntot
            phi = np.conj(fwd).T @ (v * rhot)             # sum_G v rhot exp(iG.r)
            w[j] -= occ[i] * psi[i] * phi
            ex += occ[i] * occ[j] * np.sum(v * np.abs(rhot) ** 2)
    vpsi = (w @ np.conj(e_sphere).T) * np.sqrt(vol) / ntot
    return vpsi, -0.5 * vol * ex


def fock_direct_to(c_occ, occ, c_trial, miller, grid, cell, vfun):
    """V_x phi_a on the sphere for trial orbitals, from direct sums."""
    a = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    vol = abs(np.linalg.det(a))
    pts = grid_points(grid)
    ntot = pts.shape[0]
    fr = grid_freqs(grid)
    b = recip(cell)
    g2 = np.einsum("gx,gx->g", fr @ b, fr @ b)
    v = vfun(g2)
    e_sphere = phase(np.asarray(miller), pts, grid)
    fwd = np.conj(phase(fr, pts, grid))
    psi = (c_occ @ e_sphere) / np.sqrt(vol)
    phi = (c_trial @ e_sphere) / np.sqrt(vol)
    w = np.zeros_like(phi)
    for t in range(phi.shape[0]):
        for i in range(psi.shape[0]):
            rhot = fwd @ (np.conj(psi[i]) * phi[t]) / ntot
            w[t] -= occ[i] * psi[i] * (np.conj(fwd).T @ (v * rhot))
    return (w @ np.conj(e_sphere).T) * np.sqrt(vol) / ntot
