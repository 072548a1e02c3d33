"""The boundary is a C ABI: a C11 program (``tests/c_abi_example.c``) that
includes only ``include/fock.h`` compiles with strict warnings as errors,
links against ``libfockx.so`` and gets the documented results from the
host-only entry points (the sphere, against the oracle's; the pair schedule;
status strings; the shared argument rules).  No GPU is needed."""

import os
import shutil
import subprocess

import pytest

import oracle
from tests._common import ROOT, built_library, cubic


def test_plain_c_program_uses_the_library(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    built_library()
    libdir = os.path.join(ROOT, "paper_1305_7313_gb300")
    exe = str(tmp_path / "c_abi_example")
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_example.c"), "-L" + libdir, "-lfockx",
                    "-Wl,-rpath," + libdir, "-o", exe], check=True, capture_output=True)
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout + res.stderr
    out = {line.split()[0]: line.split(None, 1)[1] for line in res.stdout.splitlines()}
    mill, _ = oracle.gsphere((24, 24, 24), cubic(10.0), 10.0)
    assert int(out["npw"]) == len(mill) == 1503
    assert [int(v) for v in out["first"].split()] == mill[0].tolist()
    assert [int(v) for v in out["last"].split()] == mill[-1].tolist()
    assert int(out["pairs"]) == 10 * 11 // 2
    assert out["status"] == "ok|the plane-wave sphere does not fit on the grid"
    assert out["failures"] == "0"
