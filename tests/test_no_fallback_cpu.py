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
