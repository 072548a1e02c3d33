"""The product path has no fallback: without ``libfockx.so`` every entry point
of the binding raises, telling the user to build, and no module of the
package imports the oracle (only the tests, ``__graft_entry__.smoke`` and the
benchmark's baseline arms may), nor does the oracle import anything of the
package.  No GPU is needed."""

import ast
import os

import pytest

from paper_1305_7313_gb300 import _lib
from tests._common import ROOT, cubic


def test_without_the_library_the_binding_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libfockx.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.fock_gsphere((24, 24, 24), cubic(10.0), 10.0)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.fock_schedule(8)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def test_the_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1305_7313_gb300")
    seen = []
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if not f.endswith(".py"):
                continue
            path = os.path.join(dirpath, f)
            seen.append(f)
            for node in ast.walk(ast.parse(open(path).read())):
                names = []
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom):
                    names = [node.module or ""]
                assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (path, names)
    assert "_lib.py" in seen and "plan.py" in seen


def test_the_oracle_imports_nothing_from_the_package():
    odir = os.path.join(ROOT, "oracle")
    for f in sorted(os.listdir(odir)):
        if not f.endswith(".py"):
            continue
        for node in ast.walk(ast.parse(open(os.path.join(odir, f)).read())):
            names = []
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom) and node.level == 0:
                names = [node.module or ""]
            for n in names:
                assert n.split(".")[0] in {"numpy", "scipy", "math", "itertools", "functools", "os"}, (f, n)


def test_orbital_tensors_are_checked_against_the_plan_before_any_device_use(monkeypatch):
    # the library takes the row length from the plan; a tensor of another
    # sphere is refused by the binding before a device pointer is formed
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(_lib, "fock_plan_npw", lambda plan: 100)
    monkeypatch.setattr(_lib, "fock_kplan_npw", lambda plan, k: 100 + k)
    monkeypatch.setattr(_lib, "fock_kplan_nk", lambda plan: 2)
    good = torch.zeros((3, 100), dtype=torch.complex128)
    bad = torch.zeros((3, 99), dtype=torch.complex128)
    occ = [2.0, 2.0, 2.0]
    calls = [
        lambda psi, v: _lib.fock_apply(None, psi, occ, v),
        lambda psi, v: _lib.fock_apply_shard(None, psi, occ, 0, 2, v),
        lambda psi, v: _lib.fock_set_occupied(None, psi, occ),
        lambda psi, v: _lib.fock_apply_fixed(None, psi, v),
        lambda psi, v: _lib.fock_pair_energies(None, psi, [(0, 1)]),
        lambda psi, v: _lib.fock_pair_energies_static(None, psi, [(0, 1)]),
        lambda psi, v: _lib.fock_batch_create([None], [psi], [occ], [v]),
    ]
    for call in calls:
        with pytest.raises(ValueError, match="plan's sphere"):
            call(bad, good)
        with pytest.raises(TypeError, match="CUDA tensor"):
            call(good, good)
    with pytest.raises(ValueError, match="plan's sphere"):  # output of the wrong shape
        _lib.fock_apply(None, good, occ, bad)
    # k points: row length per k, the same bands at every k
    k0 = torch.zeros((3, 100), dtype=torch.complex128)
    k1 = torch.zeros((3, 101), dtype=torch.complex128)
    with pytest.raises(ValueError, match="plan's sphere"):
        _lib.fock_kplan_apply(None, [k0, k0], [[2.0] * 3] * 2, [k0, k0])
    with pytest.raises(ValueError, match="plan's sphere"):
        _lib.fock_kplan_apply(None, [k0, torch.zeros((2, 101), dtype=torch.complex128)], [[2.0] * 3] * 2, [k0, k1])
    with pytest.raises(TypeError, match="CUDA tensor"):
        _lib.fock_kplan_apply(None, [k0, k1], [[2.0] * 3] * 2, [k0, k1])
    # the plan's k-point count: fewer (or more) tensor lists than k points, or
    # occupations of another shape, are refused before any pointer is formed
    with pytest.raises(ValueError, match="k points"):
        _lib.fock_kplan_apply(None, [k0], [[2.0] * 3], [k0])
    with pytest.raises(ValueError, match="k points"):
        _lib.fock_kplan_apply(None, [k0, k1, k1], [[2.0] * 3] * 3, [k0, k1, k1])
    with pytest.raises(ValueError, match="k points"):
        _lib.fock_kplan_apply(None, [k0, k1], [[2.0] * 3] * 2, [k0])
    with pytest.raises(ValueError, match="one row of occupations per k point"):
        _lib.fock_kplan_apply(None, [k0, k1], [2.0] * 6, [k0, k1])
    with pytest.raises(ValueError, match="one row of occupations per k point"):
        _lib.fock_kplan_apply(None, [k0, k1], [[2.0] * 2] * 3, [k0, k1])
