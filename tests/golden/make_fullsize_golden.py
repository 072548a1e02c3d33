"""Write ``oracle_fullsize_N96_nb64.txt``: the oracle's exchange energy, its
omega-derivative and sampled V_x psi on the first 64 bands of the two 96^3
workloads (cubic cell L = 27 bohr, Ecut = 12 Ha, 39,127 plane waves, f = 2):

* the Spencer-Alavi workload (seed 1306; the FP64 and double-float forms),
* the erfc workload at omega = 0.106 (seed 1307; the mixed form).

The 64 bands are the first rows of the full 512-band seeded set (the Loewdin
orthonormalisation runs over all 512), so the subset is the one the benchmark
and the full-size tests build.  The sums run over the 64 bands only: every
ordered pair (i, j) of them, 4,096 pairs, 2,080 unique.

The paper prints no worked numerical example of the method; these are the
oracle's own values.  Calls only ``oracle/`` and the seeded input generator
(``synth.py``, loaded from its file).  Takes a few minutes of host time.
Run from the repository root:

    python tests/golden/make_fullsize_golden.py
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

from tests.golden.fullsize_record import FILE, NB, NB_ALL  # noqa: E402  (the reader of the same file)
N, L, ECUT = 96, 27.0, 12.0
# (name, kernel, omega, seed): the seeds of the 96^3 workloads
CASES = (("spencer_alavi_seed1306", "spencer_alavi", None, 1306), ("erfc_seed1307", "erfc", 0.106, 1307))
BANDS = (0, 31, 63)           # bands whose V_x psi is sampled
STRIDE = 193                  # sphere positions 0, 193, 386, ... (203 samples of 39,127)


def compute():
    """{case: (vpsi [NB, npw], ex, dex)} and the sphere size."""
    cell = (L * np.eye(3)).ravel()
    grid = (N, N, N)
    mill, _ = oracle.gsphere(grid, cell, ECUT)
    out = {}
    for name, kind, omega, seed in CASES:
        c = synth.orbitals(mill, cell, NB_ALL, seed)[:NB]
        occ = np.full(NB, 2.0)
        out[name] = oracle.fock_apply(c, occ, mill, grid, cell, kind, omega)
    return len(mill), out


def render(npw, out):
    lines = [
        "# Oracle (FP64) results on the first 64 bands of the 96^3 / L = 27 bohr / Ecut = 12 Ha",
        "# workloads (synthetic orbitals: first 64 rows of the 512-band seeded set, f = 2):",
        "# E_x and dE_x/domega over the 64 bands, and per sampled band b the largest |V_x psi_b(G)|",
        "# over the sphere and V_x psi_b(G) at sphere positions 0, %d, %d, ..." % (STRIDE, 2 * STRIDE),
        "# The paper prints no worked example of the method; these are the oracle's own",
        "# values, written by tests/golden/make_fullsize_golden.py (oracle/ and the seeded",
        "# input generator only).",
        "npw %d nb %d" % (npw, NB),
    ]
    for name, _, _, _ in CASES:
        v, ex, dex = out[name]
        lines.append("case %s ex %.17e dex %.17e" % (name, ex, dex))
        for b in BANDS:
            lines.append("vmax %s %d %.17e" % (name, b, np.max(np.abs(v[b]))))
            for g in range(0, npw, STRIDE):
                lines.append("coef %s %d %d %.17e %.17e" % (name, b, g, v[b, g].real, v[b, g].imag))
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    npw, out = compute()
    with open(FILE, "w") as fh:
        fh.write(render(npw, out))
    print("wrote", FILE)
