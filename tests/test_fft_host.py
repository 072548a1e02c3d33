"""The transforms' in-register DFTs (``Dft`` in ``csrc/fft_core.cuh``: radices
2, 3, 4 and 8 written out, 6, 9, 12 and 16 as two small DFTs with
compile-time twiddles; plain, and with twiddled inputs whose products are
folded into the butterfly sums by fused multiply-adds) compiled for the host
by nvcc and checked against the DFT evaluated directly in FP64 on the very
values the butterflies saw; and the radix plans the kernels are compiled with
(make_radix_plan) against the stage constraints and a brute-force search.  No
GPU is needed.

Bound: a length-R DFT computed in u-precision arithmetic (float u = 2^-24,
double u = 2^-53) errs by at most a few u log2(R) times sum_r |x_r|; the
tolerances are 2e-6 (float) and 1e-14 (double) of that sum.
"""

import subprocess

import numpy as np
import pytest

from tests._common import host_program

RADICES = (2, 3, 4, 6, 8, 9, 12, 16)
TOL = {0: 2e-6, 1: 1e-14}


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    """The host driver, compiled by nvcc into a temporary folder."""
    return host_program("fft_host_driver.cu", tmp_path_factory.mktemp("fft_host"))


@pytest.fixture(scope="module")
def cases(driver):
    out = subprocess.run([driver], check=True, capture_output=True, text=True).stdout
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


# ---- radix plans (make_radix_plan, evaluated at compile time as in the kernels)

ALLOWED = (16, 12, 9, 8, 6, 4, 3, 2)


@pytest.fixture(scope="module")
def plans(driver):
    out = subprocess.run([driver, "plans"], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        f = line.split()
        n, maxt, emax, nst = (int(v) for v in f[1:5])
        radices = tuple(int(v) for v in f[5:5 + nst])
        got[(n, maxt, emax)] = (radices, int(f[9]), int(f[10]))
    return got


def _round32(t):
    return (t + 31) // 32 * 32


def _best_tl(n, radices, nlines, maxt, emax):
    """Largest sub-threads per line t that divides every stage's butterfly
    count n / r, keeps n / t elements a thread within emax and the CTA
    (nlines t, whole warps) within maxt; 0 if none."""
    ok = [t for t in range(1, n + 1)
          if all((n // r) % t == 0 for r in radices) and n // t <= emax and _round32(nlines * t) <= maxt]
    return max(ok, default=0)


def _multisets(n, max_len=4):
    """Every multiset of allowed radices (as a descending tuple) with product n."""
    out = set()

    def grow(rem, prefix):
        if rem == 1:
            out.add(tuple(sorted(prefix, reverse=True)))
            return
        if len(prefix) == max_len:
            return
        for r in ALLOWED:
            if rem % r == 0:
                grow(rem // r, prefix + [r])

    grow(n, [])
    return out


def test_radix_plans_obey_the_stage_constraints(plans):
    for (n, maxt, emax), (radices, tlp, tlc) in plans.items():
        assert 1 <= len(radices) <= 4 and int(np.prod(radices)) == n, (n, radices)
        assert all(r in ALLOWED for r in radices)
        for tl, nlines in ((tlp, n), (tlc, 2 * (n // 2 + 1))):
            assert tl >= 1
            assert all((n // r) % tl == 0 for r in radices)  # whole butterflies per thread
            assert n // tl <= emax                            # registers a thread holds
            assert _round32(nlines * tl) <= maxt              # CTA size


def test_radix_plans_take_the_fewest_stages_then_the_most_threads(plans):
    for (n, maxt, emax), (radices, tlp, tlc) in plans.items():
        valid = []
        for m in _multisets(n):
            p = _best_tl(n, m, n, maxt, emax)
            c = _best_tl(n, m, 2 * (n // 2 + 1), maxt, emax)
            if p and c:
                valid.append((len(m), -p, m, c))
        fewest = min(v[0] for v in valid)
        most = max(-v[1] for v in valid if v[0] == fewest)
        assert len(radices) == fewest and tlp == most, (n, maxt, emax, radices, tlp)
        assert tlp == _best_tl(n, radices, n, maxt, emax)
        assert tlc == _best_tl(n, radices, 2 * (n // 2 + 1), maxt, emax)


def test_the_benchmark_grids_use_the_documented_plans(plans):
    # 96: 12 x 8 with 4 threads per line in FP32, 12 x 4 x 2 with 8 in FP64 and
    # double-float; 48: 12 x 4 with 4 threads per line
    assert plans[(96, 1024, 24)] == ((12, 8), 4, 4)
    assert plans[(96, 1024, 12)] == ((12, 4, 2), 8, 8)
    assert plans[(48, 1024, 24)] == ((12, 4), 4, 4)
