"""Coulomb kernels v(G) (oracle; test infrastructure).

The paper writes the exchange kernel as 1/|G+q|^2 (§4, reciprocal-space E_x
and V_x equations) and does not treat its divergence at G = q = 0.  At the
Gamma point the finite kernels below are used, with the 4 pi of Hartree units
included:

* Spencer-Alavi spherical truncation at Rc = (3 Omega / 4 pi)^(1/3):
  v(G) = 4 pi (1 - cos(|G| Rc)) / |G|^2 = 8 pi sin^2(|G| Rc / 2) / |G|^2,
  v(0) = 2 pi Rc^2.
* erfc screening with range parameter omega (bohr^-1):
  v(G) = 4 pi (1 - exp(-|G|^2 / 4 omega^2)) / |G|^2, v(0) = pi / omega^2,
  dv/domega = -(2 pi / omega^3) exp(-|G|^2 / 4 omega^2) (G = 0 included).

Both kernels are real, non-negative and even in G.
"""

import numpy as np

SPENCER_ALAVI = "spencer_alavi"
ERFC = "erfc"


def spencer_alavi_rc(volume):
    return (3.0 * volume / (4.0 * np.pi)) ** (1.0 / 3.0)


def coulomb_kernel(kind, g2, volume, omega=None):
    """v(G) for an array of |G|^2 values."""
    g2 = np.asarray(g2, dtype=np.float64)
    v = np.empty_like(g2)
    zero = g2 == 0.0
    nz = ~zero
    if kind == SPENCER_ALAVI:
        rc = spencer_alavi_rc(volume)
        g = np.sqrt(g2[nz])
        s = np.sin(0.5 * g * rc)
        v[nz] = 8.0 * np.pi * s * s / g2[nz]
        v[zero] = 2.0 * np.pi * rc * rc
    elif kind == ERFC:
        if omega is None or omega <= 0.0:
            raise ValueError("erfc kernel needs omega > 0")
        v[nz] = -4.0 * np.pi * np.expm1(-g2[nz] / (4.0 * omega * omega)) / g2[nz]
        v[zero] = np.pi / (omega * omega)
    else:
        raise ValueError("unknown kernel kind %r" % (kind,))
    return v


def coulomb_kernel_domega(kind, g2, volume, omega=None):
    """dv/domega; zero for the Spencer-Alavi kernel, which has no omega."""
    g2 = np.asarray(g2, dtype=np.float64)
    if kind == SPENCER_ALAVI:
        return np.zeros_like(g2)
    if kind == ERFC:
        return -(2.0 * np.pi / omega**3) * np.exp(-g2 / (4.0 * omega * omega))
    raise ValueError("unknown kernel kind %r" % (kind,))
