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
