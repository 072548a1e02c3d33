"""Plain FP64 CPU oracle for the Γ-point Fock exact-exchange apply.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (the C-ABI library and its Python binding) never calls it,
and this package imports nothing from the product: the two share no code.

What it computes (the paper's §4, "The Exact Exchange (EXX) within the
planewave method"):

* E_x from overlap ("pair") charge densities M_ij(G) = FT[u_j* u_i], summed with
  the Coulomb kernel over G (the reciprocal-space E_x equation of §4); the
  printed ``M*(G) M(G')`` is read as diagonal in G.
* V_x|u_j> as the real-space product of each occupied orbital with the
  potential of the pair density (the V_x equation of §4, whose printed form is
  garbled into a scalar; the operator form used here is the standard one that
  the E_x equation differentiates to).
* Pair densities obtained by transforming orbitals to real space, multiplying
  pointwise and transforming back (the §4 paragraph on overlap charge densities
  computed by FFT).

Everything is evaluated one pair at a time, in FP64, with ``numpy.fft`` as the
only library primitive: no packing of two pairs into one transform, no fusion,
no blocking.

``oracle.sternheimer`` adds the linear-response solve of §3.1 (the Sternheimer
equation (H - eps_n + alpha P) g_n = -Q w_n by CG, with the paper's regrouping
of converged and unconverged bands) for a model Hamiltonian, kinetic energy
plus a local potential on the same plane-wave sphere.

Parity pins (see ``tests/test_oracle_*.py``): a direct O(N^2) DFT on tiny
grids, closed-form Gaussian self-energies for both kernels, Hermiticity and
negative semidefiniteness of <psi_a|V_x|psi_b>, E_x = 1/2 sum_j f_j
<psi_j|V_x psi_j>, finite differences of E_x in psi and in omega, unitary,
translation, permutation and partition invariances, and brute-force counts of
the G-sphere; for the Sternheimer solve, the model H's FFT route against the
dense matrix of the potential's Fourier coefficients (itself checked against
closed forms) and the CG solution against a direct dense solve.  No function
here is "parity unpinned".
"""

from .lattice import reciprocal_lattice, cell_volume, gsphere, gsphere_k, grid_miller, grid_g2
from .kernels import coulomb_kernel, coulomb_kernel_domega, spencer_alavi_rc
from .fock import (
    orbitals_to_real,
    real_to_sphere,
    pair_potential,
    pair_energy,
    fock_apply,
    fock_apply_to,
    fock_apply_kpoints,
    overlap_matrix_vx,
    exchange_energy_from_vpsi,
)

__all__ = [
    "reciprocal_lattice",
    "cell_volume",
    "gsphere",
    "gsphere_k",
    "grid_miller",
    "grid_g2",
    "coulomb_kernel",
    "coulomb_kernel_domega",
    "spencer_alavi_rc",
    "orbitals_to_real",
    "real_to_sphere",
    "pair_potential",
    "pair_energy",
    "fock_apply",
    "fock_apply_to",
    "fock_apply_kpoints",
    "overlap_matrix_vx",
    "exchange_energy_from_vpsi",
]
