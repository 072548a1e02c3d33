"""Seeded synthetic orbitals: the one input generator shared by tests and bench.

It holds none of the exchange arithmetic; it only draws plane-wave coefficients
with the statistics of a large-cell ground state:

1. c_n(G) = (N(0,1) + i N(0,1)) * exp(-|G|^2 / 4) on the sphere, drawn with
   ``numpy.random.default_rng(seed)`` in row-major (band, G) order;
2. Hermitian symmetrisation c(G) <- (c(G) + c(-G)*) / 2, so psi(r) is real
   (Gamma point) and c(0) is real;
3. Loewdin orthonormalisation C <- C S^-1/2 with the real overlap
   S_ab = Re sum_G c_a(G)* c_b(G), followed by one more exact symmetrisation so
   that c(-G) = c(G)* holds bit for bit.

The caller passes the sphere (Miller indices, any order) and the cell; the
coefficients come back in the same order.
"""

import numpy as np


def _recip(cell):
    a = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    return 2.0 * np.pi * np.linalg.inv(a).T


def mirror_index(miller):
    """Position of -G for every G of the list (the list must be closed under G -> -G)."""
    m = np.asarray(miller, dtype=np.int64)
    key = {tuple(r): k for k, r in enumerate(m.tolist())}
    return np.array([key[(-r[0], -r[1], -r[2])] for r in m.tolist()], dtype=np.int64)


def _symmetrise(c, mir):
    return 0.5 * (c + np.conj(c[:, mir]))


def orbitals(miller, cell, nbands, seed):
    """Orthonormal Gamma-point orbitals, complex128 array [nbands, npw]."""
    m = np.asarray(miller, dtype=np.float64)
    g = m @ _recip(cell)
    g2 = np.einsum("gx,gx->g", g, g)
    rng = np.random.default_rng(seed)
    npw = m.shape[0]
    c = rng.standard_normal((nbands, npw)) + 1j * rng.standard_normal((nbands, npw))
    c = c * np.exp(-0.25 * g2)[None, :]
    mir = mirror_index(miller)
    c = _symmetrise(c, mir)
    s = (np.conj(c) @ c.T).real
    w, u = np.linalg.eigh(s)
    x = (u * (1.0 / np.sqrt(w))[None, :]) @ u.T
    c = x.T @ c
    c = _symmetrise(c, mir)
    return np.ascontiguousarray(c)


def gaussian_orbital(miller, cell, sigma, center=(0.0, 0.0, 0.0)):
    """Plane-wave coefficients of psi(r) = (2 pi sigma^2)^-3/4 exp(-|r-R|^2 / 4 sigma^2).

    Analytic transform c(G) = Omega^-1/2 (8 pi sigma^2)^3/4 exp(-sigma^2 |G|^2)
    exp(-i G.R), renormalised on the sphere.  Used for closed-form checks.
    """
    a = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    vol = abs(np.linalg.det(a))
    g = np.asarray(miller, dtype=np.float64) @ _recip(cell)
    g2 = np.einsum("gx,gx->g", g, g)
    c = (8.0 * np.pi * sigma * sigma) ** 0.75 / np.sqrt(vol) * np.exp(-sigma * sigma * g2)
    c = c * np.exp(-1j * (g @ np.asarray(center, dtype=np.float64)))
    c = c / np.sqrt(np.sum(np.abs(c) ** 2))
    return c[None, :].astype(np.complex128)


def orbitals_k(miller, cell, kfrac, nbands, seed):
    """Orthonormal Bloch orbitals at k (reduced coordinates kfrac), complex128 [nbands, npw].

    c(G) = (N(0,1) + i N(0,1)) exp(-|k + G|^2 / 4), Loewdin-orthonormalised with
    the Hermitian overlap S = C* C^T; no symmetry between G and -G.
    """
    m = np.asarray(miller, dtype=np.float64) + np.asarray(kfrac, dtype=np.float64)[None, :]
    g = m @ _recip(cell)
    g2 = np.einsum("gx,gx->g", g, g)
    rng = np.random.default_rng(seed)
    npw = m.shape[0]
    c = rng.standard_normal((nbands, npw)) + 1j * rng.standard_normal((nbands, npw))
    c = c * np.exp(-0.25 * g2)[None, :]
    s = np.conj(c) @ c.T
    w, u = np.linalg.eigh(s)
    x = (u * (1.0 / np.sqrt(w))[None, :]) @ np.conj(u).T
    return np.ascontiguousarray(x.T @ c)


def model_potential(grid, cell, seed=7, depth=1.5, width=0.9, centers=3):
    """A real local potential V(r) on the FFT grid, float64 [N1, N2, N3]: a few
    Gaussian wells -depth exp(-|r - R|^2 / (2 width^2)) at seeded fractional
    positions R (nearest periodic image), with no symmetry that would make the
    states of H = -1/2 nabla^2 + V degenerate."""
    rng = np.random.default_rng(seed)
    a = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    idx = np.stack(np.meshgrid(*[np.arange(n) / n for n in grid], indexing="ij"), axis=-1)
    v = np.zeros(tuple(int(n) for n in grid))
    for _ in range(centers):
        f = rng.random(3)
        d = idx - f
        d -= np.round(d)
        r = d @ a
        v -= depth * np.exp(-np.einsum("...x,...x->...", r, r) / (2 * width ** 2))
    return v
