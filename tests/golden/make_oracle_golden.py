"""Write ``oracle_gamma_L10_N24_nb8.txt``: the oracle's exchange energy, its
omega-derivative and V_x psi (norms and sampled coefficients) on the smallest
workload: 24^3 grid, cubic cell L = 10 bohr, Ecut = 10 Ha, 8 bands of seeded
synthetic orbitals (seed 1305), f = 2, for the Spencer-Alavi kernel and for the
erfc kernel at omega = 0.106.

The paper prints no worked numerical example of the method (its tables are
wall-clock times and parallel efficiencies), so no stored value here is the
paper's: this file is a record of the oracle's own results, which the oracle's
pins (closed forms, brute-force DFTs, invariants) do not replace, and which any
later change to the oracle's arithmetic must reproduce or justify.

Calls only ``oracle/`` and the seeded input generator (``synth.py``, loaded
from its file).  Run from the repository root:

    python tests/golden/make_oracle_golden.py
"""

import importlib.util
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402

_spec = importlib.util.spec_from_file_location("synth", os.path.join(ROOT, "paper_1305_7313_gb300", "synth.py"))
synth = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(synth)

FILE = os.path.join(HERE, "oracle_gamma_L10_N24_nb8.txt")
N, L, ECUT, NB, SEED = 24, 10.0, 10.0, 8, 1305
KERNELS = (("spencer_alavi", None), ("erfc", 0.106))
SAMPLES = (0, 1, 7, 100, 1000)  # positions in the canonical sphere order


def compute():
    """{kernel: (vpsi [nb, npw], ex, dex)} and the sphere size."""
    cell = (L * np.eye(3)).ravel()
    grid = (N, N, N)
    mill, _ = oracle.gsphere(grid, cell, ECUT)
    c = synth.orbitals(mill, cell, NB, SEED)
    occ = np.full(NB, 2.0)
    out = {kind: oracle.fock_apply(c, occ, mill, grid, cell, kind, omega) for kind, omega in KERNELS}
    return len(mill), out


def render(npw, out):
    lines = [
        "# Oracle (FP64) results on the 24^3 / L = 10 bohr / Ecut = 10 Ha / 8-band workload",
        "# (synthetic orbitals, seed 1305, f = 2): E_x and dE_x/domega per kernel, the norm",
        "# of V_x psi_b and V_x psi_b(G) at sphere positions %s." % ", ".join(str(g) for g in SAMPLES),
        "# The paper prints no worked example of the method; these are the oracle's own",
        "# values, written by tests/golden/make_oracle_golden.py (oracle/ and the seeded",
        "# input generator only).",
        "npw %d" % npw,
    ]
    for kind, _ in KERNELS:
        v, ex, dex = out[kind]
        lines.append("kernel %s ex %.17e dex %s" % (kind, ex, "none" if dex is None else "%.17e" % dex))
        for b in range(v.shape[0]):
            lines.append("norm %s %d %.17e" % (kind, b, np.linalg.norm(v[b])))
            for g in SAMPLES:
                lines.append("coef %s %d %d %.17e %.17e" % (kind, b, g, v[b, g].real, v[b, g].imag))
    return "\n".join(lines) + "\n"


def parse(text):
    """{"npw": n, kind: {"ex", "dex", "norm": {b: x}, "coef": {(b, g): complex}}}"""
    rec = {}
    for line in text.splitlines():
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "npw":
            rec["npw"] = int(f[1])
        elif f[0] == "kernel":
            rec[f[1]] = {"ex": float(f[3]), "dex": None if f[5] == "none" else float(f[5]), "norm": {}, "coef": {}}
        elif f[0] == "norm":
            rec[f[1]]["norm"][int(f[2])] = float(f[3])
        elif f[0] == "coef":
            rec[f[1]]["coef"][(int(f[2]), int(f[3]))] = complex(float(f[4]), float(f[5]))
    return rec


if __name__ == "__main__":
    npw, out = compute()
    with open(FILE, "w") as fh:
        fh.write(render(npw, out))
    print("wrote", FILE)
