"""Cell, reciprocal lattice and plane-wave sphere (oracle; test infrastructure).

The paper expands orbitals in plane waves on a G basis (§3, §4: Bloch functions
u_nk expanded in plane waves, transformed to real space by FFT).  It fixes no
convention for the basis set; the readings used here are:

* Hartree atomic units; cell rows a1, a2, a3 in bohr; reciprocal rows b_i with
  b_i . a_j = 2 pi delta_ij.
* The basis is the sphere S = {G = m1 b1 + m2 b2 + m3 b3 : |G|^2 <= 2 Ecut}
  (Ecut in Ha, kinetic energy |G|^2/2).
* Canonical order of S: ascending FP64 |G|^2, ties broken lexicographically on
  (m1, m2, m3).  |G|^2 is evaluated with one fixed sequence of IEEE operations
  (written out below) so that any other implementation that follows the same
  sequence reproduces the order bit for bit.
* Grid index of Miller index m along an axis of length N is m mod N (numpy
  ``fftfreq`` order); the sphere must satisfy 2|m_a| < N_a.
"""

import numpy as np


def _cross(a, b):
    return np.array(
        [
            a[1] * b[2] - a[2] * b[1],
            a[2] * b[0] - a[0] * b[2],
            a[0] * b[1] - a[1] * b[0],
        ],
        dtype=np.float64,
    )


def cell_volume(cell):
    """Omega = a1 . (a2 x a3), summed left to right."""
    a = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    c = _cross(a[1], a[2])
    return float((a[0, 0] * c[0] + a[0, 1] * c[1]) + a[0, 2] * c[2])


def reciprocal_lattice(cell):
    """Rows b1, b2, b3 = (2 pi / Omega) * (a2 x a3, a3 x a1, a1 x a2)."""
    a = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    fac = (2.0 * np.pi) / cell_volume(a)
    return np.array(
        [_cross(a[1], a[2]) * fac, _cross(a[2], a[0]) * fac, _cross(a[0], a[1]) * fac],
        dtype=np.float64,
    )


def g2_of_miller(miller, recip):
    """|G|^2 for integer Miller indices, G = m1 b1 + m2 b2 + m3 b3.

    Each Cartesian component is accumulated as ((m1 b1x + m2 b2x) + m3 b3x) and
    |G|^2 = (Gx^2 + Gy^2) + Gz^2, with no fused multiply-add.
    """
    m = np.asarray(miller, dtype=np.float64)
    b = np.asarray(recip, dtype=np.float64)
    comps = []
    for x in range(3):
        comps.append((m[..., 0] * b[0, x] + m[..., 1] * b[1, x]) + m[..., 2] * b[2, x])
    return (comps[0] * comps[0] + comps[1] * comps[1]) + comps[2] * comps[2]


def gsphere(grid, cell, ecut):
    """Miller indices of the sphere |G|^2 <= 2*Ecut in canonical order.

    Returns ``(miller[npw, 3] int32, g2[npw] float64)``.  Raises ValueError when
    the sphere does not fit on the grid (2|m_a| must be < N_a).
    """
    grid = [int(n) for n in grid]
    b = reciprocal_lattice(cell)
    # Bound on |m_a|: |m_a| = |G . a_a| / (2 pi) <= |G| |a_a| / (2 pi).
    a = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    gmax = np.sqrt(2.0 * ecut)
    mmax = [int(np.floor(gmax * np.linalg.norm(a[i]) / (2.0 * np.pi))) + 1 for i in range(3)]
    r = [np.arange(-mm, mm + 1) for mm in mmax]
    m1, m2, m3 = np.meshgrid(r[0], r[1], r[2], indexing="ij")
    mill = np.stack([m1.ravel(), m2.ravel(), m3.ravel()], axis=1)
    g2 = g2_of_miller(mill, b)
    keep = g2 <= 2.0 * ecut
    mill = mill[keep]
    g2 = g2[keep]
    for ax in range(3):
        if mill.size and 2 * int(np.abs(mill[:, ax]).max()) >= grid[ax]:
            raise ValueError("G-sphere does not fit on the FFT grid")
    order = np.lexsort((mill[:, 2], mill[:, 1], mill[:, 0], g2))
    return mill[order].astype(np.int32), g2[order]


def grid_miller(grid):
    """Miller index of every grid point, numpy fftfreq order, shape (3, N1, N2, N3)."""
    axes = [np.fft.fftfreq(int(n), d=1.0 / int(n)).round().astype(np.int64) for n in grid]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=0)


def grid_g2(grid, cell):
    """|G|^2 on every point of the full FFT grid (fftfreq order)."""
    m = grid_miller(grid)
    return g2_of_miller(np.moveaxis(m, 0, -1), reciprocal_lattice(cell))


def g2_of_miller_k(miller, recip, kfrac):
    """|k + G|^2 with k = kf1 b1 + kf2 b2 + kf3 b3 (reduced coordinates).

    Each Cartesian component is ((m1 + kf1) b1x + (m2 + kf2) b2x) + (m3 + kf3) b3x,
    the sum m + kf formed first; kf = 0 gives exactly g2_of_miller.
    """
    m = np.asarray(miller, dtype=np.float64)
    k = np.asarray(kfrac, dtype=np.float64)
    b = np.asarray(recip, dtype=np.float64)
    u = [m[..., a] + k[a] for a in range(3)]
    comps = [(u[0] * b[0, x] + u[1] * b[1, x]) + u[2] * b[2, x] for x in range(3)]
    return (comps[0] * comps[0] + comps[1] * comps[1]) + comps[2] * comps[2]


def gsphere_k(grid, cell, ecut, kfrac):
    """Miller indices of {G : |k + G|^2 <= 2 Ecut} in canonical order
    (ascending FP64 |k + G|^2, ties lexicographic on (m1, m2, m3))."""
    grid = [int(n) for n in grid]
    b = reciprocal_lattice(cell)
    a = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    gmax = np.sqrt(2.0 * ecut)
    kf = np.asarray(kfrac, dtype=np.float64)
    mmax = [int(np.floor(gmax * np.linalg.norm(a[i]) / (2.0 * np.pi) + abs(kf[i]))) + 1 for i in range(3)]
    r = [np.arange(-mm, mm + 1) for mm in mmax]
    m1, m2, m3 = np.meshgrid(r[0], r[1], r[2], indexing="ij")
    mill = np.stack([m1.ravel(), m2.ravel(), m3.ravel()], axis=1)
    g2 = g2_of_miller_k(mill, b, kf)
    keep = g2 <= 2.0 * ecut
    mill, g2 = mill[keep], g2[keep]
    for ax in range(3):
        if mill.size and 2 * int(np.abs(mill[:, ax]).max()) >= grid[ax]:
            raise ValueError("G-sphere does not fit on the FFT grid")
    order = np.lexsort((mill[:, 2], mill[:, 1], mill[:, 0], g2))
    return mill[order].astype(np.int32), g2[order]
