"""The Coulomb kernels the plans tabulate (``kernel_value`` in
``csrc/fock_lattice.h``: Spencer-Alavi truncation and erfc screening, their
G = 0 limits and dv/domega) against the oracle's kernels, which the oracle's
own pins tie to radial quadrature and closed forms.  Both evaluate the same
FP64 expressions (Rc by cbrt in the library, by a cube-root power in the
oracle), so they agree to a few units in the last place of what the kernels'
conditioning allows: erfc, and Spencer-Alavi at G = 0, to 1e-14 relative;
Spencer-Alavi, v = 8 pi sin^2(x) / |G|^2 with x = |G| Rc / 2, to 1e-14 of
(8 pi / |G|^2) * 2x, the change an error of one part in 1e16 of x makes (near
the zeros of sin, where v itself is small, a relative bound would not hold).
Host code only: no GPU."""

import subprocess

import numpy as np
import pytest

from oracle.kernels import ERFC, SPENCER_ALAVI, coulomb_kernel, coulomb_kernel_domega
from tests._common import host_program

RTOL = 1e-14


@pytest.fixture(scope="module")
def values(tmp_path_factory):
    exe = host_program("lattice_host_driver.cpp", tmp_path_factory.mktemp("lattice_host"))
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = [line.split() for line in out.splitlines()]
    return [(int(r[0]), *(float.fromhex(x) for x in r[1:])) for r in rows]


def test_kernels_match_the_oracle(values):
    assert len(values) == 5 * 16 * 5
    for kind, vol, omega, g2, v, dv in values:
        okind = SPENCER_ALAVI if kind == 0 else ERFC
        om = None if kind == 0 else omega
        ref = coulomb_kernel(okind, np.array([g2]), vol, om)[0]
        dref = coulomb_kernel_domega(okind, np.array([g2]), vol, om)[0]
        assert v > 0.0
        if kind == 0 and g2 > 0.0:
            x = 0.5 * np.sqrt(g2) * (3.0 * vol / (4.0 * np.pi)) ** (1.0 / 3.0)
            scale = 8.0 * np.pi / g2 * max(1.0, 2.0 * x)
        else:
            scale = abs(ref)
        assert abs(v - ref) <= RTOL * scale, (kind, vol, omega, g2)
        assert abs(dv - dref) <= RTOL * abs(dref), (kind, vol, omega, g2)


def test_the_g0_values_are_the_limits(values):
    for kind, vol, omega, g2, v, dv in values:
        if g2 == 0.0:
            rc = (3.0 * vol / (4.0 * np.pi)) ** (1.0 / 3.0)
            lim = 2.0 * np.pi * rc * rc if kind == 0 else np.pi / omega ** 2
            assert abs(v - lim) <= RTOL * lim
        elif g2 == 1e-12:
            # continuous at G = 0: the smallest |G|^2 lies on the limit
            zero = [x for x in values if x[:3] == (kind, vol, omega) and x[3] == 0.0][0]
            assert abs(v - zero[4]) <= 1e-9 * zero[4]
