"""The Fock exchange apply and exchange energy, one pair at a time (oracle).

Conventions (Hartree units; Omega = cell volume; the grid has Ntot = N1 N2 N3
points r_k; ``fft`` is the unnormalised forward transform with exp(-i G.r) and
``ifft`` carries the 1/Ntot):

  psi_n(r)     = Omega^-1/2 sum_{G in S} c_n(G) exp(i G.r)
               = (Ntot / sqrt(Omega)) ifft(scatter(c_n))
  rho_ij(r)    = psi_i*(r) psi_j(r)                      (overlap density, §4)
  rhot_ij(G)   = fft(rho_ij)(G) / Ntot                   (M_ij of §4)
  phi_ij(r)    = ifft(v * fft(rho_ij))(r)
  (V_x psi_j)(r) = - sum_i f_i psi_i(r) phi_ij(r)        (V_x equation of §4)
  (V_x psi_j)(G) = (sqrt(Omega) / Ntot) fft(V_x psi_j)(G),  G in S
  E_x          = -(Omega/2) sum_{i,j} f_i f_j sum_G v(G) |rhot_ij(G)|^2
                                                         (reciprocal E_x, §4)
  dE_x/domega  = -(Omega/2) sum_{i,j} f_i f_j sum_G dv/domega |rhot_ij(G)|^2

Readings of the paper used here: the printed M*(G) M(G') is diagonal in G; no
spin or occupation factor is printed, so the occupations f_i enter exactly as
above (f = 2 gives twice the spin-restricted physical value); V_x psi is
projected back onto the sphere S.  All sums over i run over every band, and the
pair loop visits every ordered pair (i, j) with its own transforms.
"""

import numpy as np

from .lattice import cell_volume, grid_g2
from .kernels import coulomb_kernel, coulomb_kernel_domega

try:  # both are library FFTs; scipy's can use several host threads
    import scipy.fft as _sfft

    def _fftn(x):
        return _sfft.fftn(x, workers=-1)

    def _ifftn(x):
        return _sfft.ifftn(x, workers=-1)

except ImportError:  # pragma: no cover
    def _fftn(x):
        return np.fft.fftn(x)

    def _ifftn(x):
        return np.fft.ifftn(x)


def _grid_index(miller, grid):
    return tuple(np.asarray(miller)[:, a] % int(grid[a]) for a in range(3))


def orbitals_to_real(c, miller, grid, cell, real=False):
    """psi_n(r) on the grid for each row c_n(G) of ``c`` (shape nb x npw).

    ``real=True`` keeps only the real part, which is the whole orbital when the
    coefficients satisfy c(-G) = c(G)* (Gamma-point real orbitals).
    """
    grid = tuple(int(n) for n in grid)
    c = np.atleast_2d(np.asarray(c, dtype=np.complex128))
    ntot = grid[0] * grid[1] * grid[2]
    scale = ntot / np.sqrt(cell_volume(cell))
    idx = _grid_index(miller, grid)
    out = np.empty((c.shape[0],) + grid, dtype=np.float64 if real else np.complex128)
    for n in range(c.shape[0]):
        box = np.zeros(grid, dtype=np.complex128)
        box[idx] = c[n]
        p = _ifftn(box) * scale
        out[n] = p.real if real else p
    return out


def real_to_sphere(f, miller, grid, cell):
    """(sqrt(Omega)/Ntot) fft(f) sampled on the sphere: the G-coefficients of f."""
    grid = tuple(int(n) for n in grid)
    ntot = grid[0] * grid[1] * grid[2]
    scale = np.sqrt(cell_volume(cell)) / ntot
    idx = _grid_index(miller, grid)
    f = np.asarray(f)
    if f.ndim == 3:
        return _fftn(f)[idx] * scale
    return np.stack([_fftn(fn)[idx] * scale for fn in f])


def kernel_grid(kind, grid, cell, omega=None):
    """v(G) and dv/domega on every point of the full grid."""
    g2 = grid_g2(grid, cell)
    vol = cell_volume(cell)
    return coulomb_kernel(kind, g2, vol, omega), coulomb_kernel_domega(kind, g2, vol, omega)


def pair_potential(psi_i, psi_j, vgrid):
    """phi_ij = ifft(v * fft(psi_i* psi_j))."""
    return _ifftn(vgrid * _fftn(np.conj(psi_i) * psi_j))


def pair_energy(psi_i, psi_j, vgrid, dvgrid=None):
    """e_ij = sum_G v(G) |rhot_ij(G)|^2 (and the same sum with dv/domega)."""
    rho = np.conj(psi_i) * psi_j
    rt = _fftn(rho) / rho.size
    w = (rt * np.conj(rt)).real
    e = float(np.sum(vgrid * w))
    if dvgrid is None:
        return e
    return e, float(np.sum(dvgrid * w))


def fock_apply(c, occ, miller, grid, cell, kind, omega=None, out_bands=None, real=True,
               psi=None, src_bands=None):
    """V_x psi_j on the sphere for j in ``out_bands`` (default: all bands).

    Returns ``(vpsi[len(out_bands), npw], ex, dex)``.  ``ex`` and ``dex`` are the
    exchange energy and its omega-derivative over the pairs visited; they are
    returned only when ``out_bands`` covers all bands (else None).
    ``src_bands`` restricts the sum over i (default: every band); summing the
    results over a partition of the bands gives the full result, which is the
    band-group distribution of the paper (§5, the EXX loop of Fig. 3).
    ``psi`` may pass precomputed real-space orbitals (from ``orbitals_to_real``).
    """
    grid = tuple(int(n) for n in grid)
    c = np.atleast_2d(np.asarray(c, dtype=np.complex128))
    occ = np.asarray(occ, dtype=np.float64)
    nb = c.shape[0]
    if psi is None:
        psi = orbitals_to_real(c, miller, grid, cell, real=real)
    vgrid, dvgrid = kernel_grid(kind, grid, cell, omega)
    ntot = grid[0] * grid[1] * grid[2]
    vol = cell_volume(cell)
    all_bands = out_bands is None
    out_bands = list(range(nb)) if all_bands else list(out_bands)
    src_bands = range(nb) if src_bands is None else list(src_bands)
    vpsi = np.empty((len(out_bands), len(miller)), dtype=np.complex128)
    esum = 0.0
    dsum = 0.0
    for a, j in enumerate(out_bands):
        acc = np.zeros(grid, dtype=psi.dtype)
        for i in src_bands:
            rho = np.conj(psi[i]) * psi[j]
            rho_g = _fftn(rho)
            phi = _ifftn(vgrid * rho_g)
            acc -= occ[i] * psi[i] * (phi.real if real else phi)
            if all_bands:
                w = (rho_g * np.conj(rho_g)).real / (ntot * ntot)
                esum += occ[i] * occ[j] * float(np.sum(vgrid * w))
                dsum += occ[i] * occ[j] * float(np.sum(dvgrid * w))
        vpsi[a] = real_to_sphere(acc, miller, grid, cell)
    if not all_bands:
        return vpsi, None, None
    return vpsi, -0.5 * vol * esum, -0.5 * vol * dsum


def fock_apply_to(c_occ, occ, c_trial, miller, grid, cell, kind, omega=None, real=True):
    """V_x phi_a for trial orbitals phi_a, with V_x defined by the occupied set.

    (V_x phi_a)(r) = - sum_i f_i psi_i(r) ifft(v fft(psi_i* phi_a))(r): the
    operator of the V_x equation of §4 applied to a function that is not one
    of the occupied orbitals, as in the inner loop of the paper's nested SCF
    (V_x fixed while the Kohn-Sham orbitals converge).  Returns [nt, npw].
    """
    grid = tuple(int(n) for n in grid)
    occ = np.asarray(occ, dtype=np.float64)
    psi = orbitals_to_real(c_occ, miller, grid, cell, real=real)
    phi = orbitals_to_real(c_trial, miller, grid, cell, real=real)
    vgrid, _ = kernel_grid(kind, grid, cell, omega)
    out = np.empty((phi.shape[0], len(miller)), dtype=np.complex128)
    for a in range(phi.shape[0]):
        acc = np.zeros(grid, dtype=phi.dtype)
        for i in range(psi.shape[0]):
            pot = _ifftn(vgrid * _fftn(np.conj(psi[i]) * phi[a]))
            acc -= occ[i] * psi[i] * (pot.real if real else pot)
        out[a] = real_to_sphere(acc, miller, grid, cell)
    return out


def overlap_matrix_vx(c, vpsi):
    """M_ab = <psi_a | V_x psi_b> = sum_G c_a(G)* (V_x psi_b)(G)."""
    return np.conj(np.asarray(c)) @ np.asarray(vpsi).T


def exchange_energy_from_vpsi(c, occ, vpsi):
    """E_x = 1/2 sum_j f_j <psi_j | V_x psi_j>."""
    d = np.einsum("jg,jg->j", np.conj(np.asarray(c)), np.asarray(vpsi)).real
    return 0.5 * float(np.dot(np.asarray(occ, dtype=np.float64), d))


def fock_apply_kpoints(c_list, occ, miller_list, kfrac, weights, grid, cell, kind, omega=None):
    """V_x psi_nk and E_x with Brillouin-zone sampling (the first two equations of §4).

    Bloch orbitals psi_nk(r) = exp(i k.r) u_nk(r), with
    psi_nk(r) = Omega^-1/2 sum_{G in S_k} c_nk(G) exp(i (k + G).r).  With q = k - k':
      rho(r)      = u_{mk'}*(r) u_{nk}(r)
      phi(r)      = ifft(v(G + q) fft(rho))(r)
      W_nk(r)     = - sum_k' w_k' sum_m f_mk' u_mk'(r) phi(r)    (periodic part of V_x psi_nk)
      (V_x psi_nk)(G) = (sqrt(Omega)/Ntot) fft(W_nk)(G),  G in S_k
      E_x = -(Omega/2) sum_{k,k'} w_k w_k' sum_{n,m} f_nk f_mk' sum_G v(G + q) |fft(rho)(G)/Ntot|^2
    ``c_list[k]``: [nb, npw_k]; ``occ``: [nk, nb]; ``miller_list[k]``: the sphere S_k;
    ``kfrac``: [nk, 3] reduced coordinates; ``weights``: [nk].  Every ordered
    pair of states is evaluated with its own transforms.  Returns (list of
    [nb, npw_k] arrays, E_x).
    """
    from .lattice import reciprocal_lattice, g2_of_miller_k
    grid = tuple(int(n) for n in grid)
    nk = len(c_list)
    occ = np.asarray(occ, dtype=np.float64).reshape(nk, -1)
    w = np.asarray(weights, dtype=np.float64)
    kf = np.asarray(kfrac, dtype=np.float64).reshape(nk, 3)
    vol = cell_volume(cell)
    b = reciprocal_lattice(cell)
    ntot = grid[0] * grid[1] * grid[2]
    u = [orbitals_to_real(c_list[k], miller_list[k], grid, cell, real=False) for k in range(nk)]
    from .lattice import grid_miller
    gm = np.moveaxis(grid_miller(grid), 0, -1)
    out = []
    esum = 0.0
    for k in range(nk):
        nb = u[k].shape[0]
        vk = np.empty((nb, len(miller_list[k])), dtype=np.complex128)
        for n in range(nb):
            acc = np.zeros(grid, dtype=np.complex128)
            for kp in range(nk):
                vq = coulomb_kernel(kind, g2_of_miller_k(gm, b, kf[k] - kf[kp]), vol, omega)
                for m in range(u[kp].shape[0]):
                    rho_g = _fftn(np.conj(u[kp][m]) * u[k][n])
                    acc -= w[kp] * occ[kp, m] * u[kp][m] * _ifftn(vq * rho_g)
                    esum += w[k] * w[kp] * occ[k, n] * occ[kp, m] * float(
                        np.sum(vq * (rho_g * np.conj(rho_g)).real)) / (ntot * ntot)
            vk[n] = real_to_sphere(acc, miller_list[k], grid, cell)
        out.append(vk)
    return out, -0.5 * vol * esum
