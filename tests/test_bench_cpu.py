"""The benchmark's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the keys of the benchmark contract."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--ref-bands", "2"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ["impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"]:
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "gamma_fp64_L27_N96_nb512"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "3 unique pairs" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_every_function_the_benchmark_calls_is_defined_or_imported():
    # the GPU legs of bench.py cannot run here; at least their calls must resolve
    import ast
    import builtins
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    known = set(dir(builtins))
    for n in ast.walk(tree):
        if isinstance(n, (ast.FunctionDef, ast.ClassDef)):
            known.add(n.name)
        elif isinstance(n, ast.Import):
            known.update((a.asname or a.name).split(".")[0] for a in n.names)
        elif isinstance(n, ast.ImportFrom):
            known.update(a.asname or a.name for a in n.names)
        elif isinstance(n, ast.Assign):
            known.update(t.id for t in n.targets if isinstance(t, ast.Name))
    called = {n.func.id for n in ast.walk(tree) if isinstance(n, ast.Call) and isinstance(n.func, ast.Name)}
    assert called <= known, sorted(called - known)


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Plan:
    grid = (96, 96, 96)

    def __init__(self, kept_fraction=0.6014030612244898):
        self.total = 96 * 2 * 49
        self.kept = round(kept_fraction * self.total)

    def columns(self):
        return self.kept, self.total


def _res(dom_ms, launches=10, chains=380):
    phases = {"pair_fwd": 1.0, "pair_col": 1.0, "pair_inv": dom_ms}
    return {"phase_ms": phases, "clocks": {"sm_mhz": 2070.0},
            "stats": {"phase_launches": {k: launches for k in phases}, "chains": chains}}


def test_roofline_arithmetic_matches_the_documented_figures():
    # the per-unit figures the design quotes, computed by the code that reports them
    import numpy as np
    b = _bench_module()
    peaks = {"hbm_gbs": 6688.8}
    # FP64: 5 n log2 n per line; per pair (fwd + col + inv) / 2 = 88.0 MFLOP at
    # 96^3 (87.4 without the column pass's two extra stored half-columns)
    r = b.roofline("fp64", _Plan(), _res(10.0), 1, peaks, "measured")
    n3, lg = 96.0 ** 3, np.log2(96)
    per_pair = (5 * n3 * 2 * lg * 2 + 2 * 5 * n3 * lg * 98 / 96) / 2
    assert abs(per_pair / 1e6 - 88.0) < 0.05
    assert abs(5 * n3 * np.log2(n3) / 1e6 - 87.4) < 0.05
    # the measured DFMA-loop rate (1.2557 TFLOP/s at 2070 MHz) is the FP64 denominator
    assert r["kernel"] == "pair_inv" and abs(r["peak"] - 1.2557) < 1e-9
    assert abs(r["achieved"] - 5 * n3 * 2 * lg * 38 / 1e-3 / 1e12) < 1e-9  # 38 chains in 1 ms
    assert abs(r["traffic"] / 1e6 - 47.18 * 38) < 1e-6  # band block 16: the capture's 47.18 MB per chain
    r4 = b.roofline("fp64", _Plan(), _res(10.0), 1, peaks, "measured", band_block=4)
    assert r4["traffic"] is None  # band block 4: not captured
    r8 = b.roofline("fp64", _Plan(), _res(10.0), 1, peaks, "measured", band_block=8)
    assert abs(r8["traffic"] / 1e6 - 54.04 * 38) < 1e-6  # the ncu capture's 2053.5 MB per 38-chain launch
    # double-float peak: the measured FP32 FMA rate (78.52 TFLOP/s = 39.26 T
    # instructions/s) / 9.4 instructions per flop
    rd = b.roofline("df64", _Plan(), _res(10.0), 1, peaks, "measured")
    assert abs(rd["peak"] - 4.177) < 0.001
    # mixed: kept half spectrum 4.34 MB; inverse pass 9.65 MB per chain at band block 8
    rm = b.roofline("mixed32", _Plan(), _res(10.0), 1, peaks, "measured", band_block=8)
    hbytes = 96 * 96 * 98 * 8.0 * _Plan().kept / _Plan().total
    assert abs(hbytes / 1e6 - 4.34) < 0.01
    assert abs(rm["bytes_per_chain"] / 1e6 - 9.65) < 0.01 and rm["bound"] == "hbm"
    assert abs(rm["traffic"] / 1e6 - 12.61 * 38) < 1e-6


def test_loop_roofline_counts_all_three_pair_passes():
    # launches on several streams: the three passes' work over the pair loop's
    # time (the step minus the phases on the call's stream)
    b = _bench_module()
    peaks = {"hbm_gbs": 6688.8}
    res = {"ms": 1000.0, "phase_ms": {"to_real": 10.0, "to_sphere": 20.0, "energy": 0.0, "pair_fwd": 500.0,
                                      "pair_col": 600.0, "pair_inv": 700.0},
           "clocks": {"sm_mhz": 2070.0}, "stats": {"chains": 1000, "phase_launches": {}}}
    r = b.roofline("fp64", _Plan(), res, 1, peaks, "measured", 8, streams=3)
    assert r["ms_pair_loop"] == 970.0 and "3 streams" in r["kernel"]
    n3 = 96.0 ** 3
    per_chain = 5 * n3 * 2 * 6.584962500721156 * 2 + 2 * 5 * n3 * 6.584962500721156 * 98 / 96
    assert abs(per_chain / 1e6 - 175.9) < 0.1  # 88.0 MFLOP per pair
    assert abs(r["achieved"] - per_chain * 1000 / 0.97 / 1e12) < 1e-9
    rm = b.roofline("mixed32", _Plan(), res, 1, peaks, "measured", 8, streams=2)
    assert abs(rm["bytes_per_chain"] / 1e6 - 24.44) < 0.05  # 4 x 4.34 MB of kept columns + 16 planes / 8
    assert abs(rm["achieved"] - rm["bytes_per_chain"] * 1000 / 0.97 / 1e9) < 1e-6
    # the mixed column pass changed after its capture: no measured loop traffic
    assert rm["traffic"] is None
    assert abs(r["traffic"] / 1e6 - 95.61 * 1000) < 1e-6  # FP64, all three kernels, 1000 chains
    assert b.roofline("fp64", _Plan(), res, 1, peaks, "measured", 4, streams=2)["traffic"] is None


def test_golden_errors_only_for_the_full_band_set():
    # the stored oracle values are for the first 64 bands of the seeded
    # 512-band set; a run over another band count builds a different set
    sys.path.insert(0, ROOT)
    import bench

    class Plan:
        grid = (96, 96, 96)

    for nb in (64, 128, 511):
        w = dict(bench.workload("gamma_fp64_L27_N96_nb512"), nb=nb)
        assert bench.golden_errors(Plan(), None, w) is None
