"""The double-float arithmetic of the double-float form (``csrc/df64.cuh``),
compiled for the host and checked in exact rational arithmetic:

* df64(d) splits a double into hi = fl32(d), lo = fl32(d - hi): error at most
  u^2 |d| with u = 2^-24;
* the sum (TwoSum of the high parts, Knuth; low parts added; FastTwoSum
  renormalisation, Dekker) errs by at most a small multiple of u^2 (|a| + |b|)
  and returns a normalised pair (hi = fl32(hi + lo));
* the product (TwoProd by a fused multiply-add, the lo * lo term dropped)
  errs by at most a small multiple of u^2 |a b|;
* scaling by a power of two is exact;
* the integer-only float-to-double conversion is exact for normal floats and
  gives 0 for zeros and subnormals.

No GPU is needed: nvcc compiles the header for the host (contraction off)."""

import subprocess
from fractions import Fraction

import numpy as np
import pytest

from tests._common import host_program

U2 = Fraction(1, 2 ** 48)  # u^2 for u = 2^-24
ADD_BOUND = 4   # multiples of u^2 (|a| + |b|)
MUL_BOUND = 8   # multiples of u^2 |a b|


@pytest.fixture(scope="module")
def records(tmp_path_factory):
    exe = host_program("df64_host_driver.cu", tmp_path_factory.mktemp("df64_host"))
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    recs = {}
    for line in out.splitlines():
        f = line.split()
        recs.setdefault(f[0], []).append([float.fromhex(v) for v in f[1:]])
    return recs


def F(x):
    return Fraction(x)


def is_float32(x):
    return float(np.float32(x)) == x


def normalised(hi, lo):
    return is_float32(hi) and is_float32(lo) and np.float32(hi) + np.float32(lo) == np.float32(hi)


def test_the_driver_ran_every_kind(records):
    assert {k: len(v) for k, v in records.items()} == {"split": 2000, "add": 4000, "sub": 4000, "mul": 4000,
                                                       "scale": 200, "conv": 514}


def test_split_of_a_double(records):
    for d, hi, lo in records["split"]:
        assert normalised(hi, lo)
        assert abs(F(hi) + F(lo) - F(d)) <= U2 * abs(F(d))


@pytest.mark.parametrize("op", ["add", "sub"])
def test_sum_and_difference(records, op):
    worst = Fraction(0)
    for ahi, alo, bhi, blo, rhi, rlo in records[op]:
        a, b = F(ahi) + F(alo), F(bhi) + F(blo)
        exact = a + b if op == "add" else a - b
        assert normalised(rhi, rlo)
        scale = abs(a) + abs(b)
        if scale:
            worst = max(worst, abs(F(rhi) + F(rlo) - exact) / (U2 * scale))
    assert worst <= ADD_BOUND, float(worst)


def test_product(records):
    worst = Fraction(0)
    for ahi, alo, bhi, blo, rhi, rlo in records["mul"]:
        exact = (F(ahi) + F(alo)) * (F(bhi) + F(blo))
        assert normalised(rhi, rlo)
        if exact:
            worst = max(worst, abs(F(rhi) + F(rlo) - exact) / (U2 * abs(exact)))
    assert worst <= MUL_BOUND, float(worst)


def test_power_of_two_scaling_is_exact(records):
    for ahi, alo, p2, rhi, rlo in records["scale"]:
        assert F(rhi) + F(rlo) == (F(ahi) + F(alo)) * F(p2)


def test_float_to_double_conversion(records):
    tiny = 2.0 ** -126  # smallest normal float
    for f, d in records["conv"]:
        if f == 0.0 or abs(f) < tiny:
            assert d == 0.0
        else:
            assert d == f
