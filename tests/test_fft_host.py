"""The transforms' in-register DFTs (``Dft`` in ``csrc/fft_core.cuh``: radices
2, 3, 4 and 8 written out, 6, 9, 12 and 16 as two small DFTs with
compile-time twiddles; plain, and with twiddled inputs whose products are
folded into the butterfly sums by fused multiply-adds) compiled for the host
by nvcc and checked against the DFT evaluated directly in FP64 on the very
values the butterflies saw.  No GPU is needed.

Bound: a length-R DFT computed in u-precision arithmetic (float u = 2^-24,
double u = 2^-53) errs by at most a few u log2(R) times sum_r |x_r|; the
tolerances are 2e-6 (float) and 1e-14 (double) of that sum.
"""

import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1305_7313_gb300", "csrc")
RADICES = (2, 3, 4, 6, 8, 9, 12, 16)
TOL = {0: 2e-6, 1: 1e-14}


def _nvcc():
    for home in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if home and os.path.exists(os.path.join(home, "bin", "nvcc")):
            return os.path.join(home, "bin", "nvcc")
    return shutil.which("nvcc")


@pytest.fixture(scope="module")
def cases(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("fft_host") / "driver")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I" + CSRC, "-I" + os.path.join(ROOT, "include"),
                    os.path.join(HERE, "fft_host_driver.cu"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    parsed = []
    for line in out.splitlines():
        f = line.split()
        typ, R, sign, mode = (int(v) for v in f[:4])
        v = np.array([float(t) for t in f[4:]])
        assert v.size == 6 * R
        z = v[0::2] + 1j * v[1::2]
        parsed.append((typ, R, sign, mode, z[:R], z[R:2 * R], z[2 * R:]))
    return parsed


def direct_dft(x, sign):
    R = x.size
    r = np.arange(R)
    return np.exp(sign * 2j * np.pi * np.outer(r, r) / R) @ x


def effective_input(x, w, mode):
    if mode == 0:
        return x
    xe = x * w
    if mode == 1:
        xe[0] = x[0]  # x_0 carries no twiddle
    return xe


def test_every_case_was_run(cases):
    seen = {(typ, R, sign, mode) for typ, R, sign, mode, *_ in cases}
    assert seen == {(t, R, s, m) for t in (0, 1) for R in RADICES for s in (-1, 1) for m in (0, 1, 2)}


def test_butterflies_match_the_direct_dft(cases):
    worst = {}
    for typ, R, sign, mode, x, w, y in cases:
        xe = effective_input(x, w, mode)
        err = np.max(np.abs(y - direct_dft(xe, sign))) / np.sum(np.abs(xe))
        key = (typ, R, sign, mode)
        worst[key] = max(worst.get(key, 0.0), err)
    bad = {k: e for k, e in worst.items() if e > TOL[k[0]]}
    assert not bad, bad


def test_the_check_tells_the_signs_and_the_twiddles_apart(cases):
    # the same comparison against a wrong reference (opposite sign, or the
    # twiddles left out) fails by far, so a dropped term or a sign slip in a
    # butterfly cannot pass the check above
    for typ, R, sign, mode, x, w, y in cases:
        xe = effective_input(x, w, mode)
        scale = np.sum(np.abs(xe))
        if R >= 3:
            assert np.max(np.abs(y - direct_dft(xe, -sign))) / scale > 1e-3
        if mode > 0:
            assert np.max(np.abs(y - direct_dft(x, sign))) / scale > 1e-3
