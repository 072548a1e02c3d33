"""Shared helpers of the test suite (inputs and the library handle)."""

import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cubic(L):
    return (float(L) * np.eye(3)).ravel()


def declared_functions():
    """Names of the functions include/fock.h declares."""
    text = open(os.path.join(ROOT, "include", "fock.h")).read()
    return re.findall(r"^(?:fock_status|const char\*)\s+(\w+)\(", text, flags=re.M)


def built_library():
    """Build libfockx.so if needed and return the loaded ctypes handle."""
    from paper_1305_7313_gb300 import build as b
    from paper_1305_7313_gb300 import _lib
    b.build()
    return _lib.load()


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_library()
    return torch


def rel_inf(a, b):
    """max |a - b| / max |b|."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def host_program(source, exe_dir, extra=()):
    """Compile a host-only test program from tests/<source> with nvcc (the
    kernels' headers compile for the host as well) and return its path; skip
    when nvcc is not available."""
    import shutil
    import subprocess
    nvcc = None
    for home in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if home and os.path.exists(os.path.join(home, "bin", "nvcc")):
            nvcc = os.path.join(home, "bin", "nvcc")
            break
    nvcc = nvcc or shutil.which("nvcc")
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = os.path.join(str(exe_dir), os.path.splitext(source)[0])
    csrc = os.path.join(ROOT, "paper_1305_7313_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off", "-I" + csrc,
                    "-I" + os.path.join(ROOT, "include"), *extra, os.path.join(ROOT, "tests", source), "-o", exe],
                   check=True, capture_output=True)
    return exe
