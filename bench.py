"""Throughput of the Fock exchange apply on one GB300 (and N GPUs under torchrun).

Default workload: Gamma-point FP64 apply, cubic cell L = 27 bohr, 96^3 grid,
Ecut = 12 Ha (39,127 plane waves), 512 bands, f = 2, Spencer-Alavi kernel: all
131,328 unique band pairs per step.  The same 96^3 / 512-band apply in the
mixed form (complex64 transforms, erfc kernel, omega = 0.106) is measured too
and reported under "mixed32".  Inputs are seeded synthetic orbitals.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "band pairs/s for Vx·ψ at 96³/512 bands, FP32 vs FP64 form; HBM % of peak"
UNIT = "band pairs/s"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP64 rate of GB300, measured: a loop of independent DFMA chains over every
# SM (csrc/probe_fma_peak.cu) runs 1.2557 TFLOP/s at the 2070 MHz maximum SM
# clock, 99.8% of the unit count (2 FP64 FMA per SM per clock over 152 SMs).
FP64_PEAK_TFLOPS = 1.2557
FP64_FLOPS_PER_CLK = FP64_PEAK_TFLOPS * 1e12 / 2.070e9
# Double-float form: the same probe's FP32 FMA loop runs 78.52 TFLOP/s (39.26 T
# FP32 instructions/s) at 2070 MHz; a double-float add costs 11 FP32
# instructions, a multiply 7, so the radix-2 mix of the 5 n log2 n count (6
# adds, 4 multiplies per 10 flops) costs 9.4 FP32 instructions per flop.
FP32_FMA_PEAK_TFLOPS = 78.52
DF64_FLOPS_PER_CLK = FP32_FMA_PEAK_TFLOPS / 2 * 1e12 / 2.070e9 / 9.4


def workload(name):
    from paper_1305_7313_gb300.workloads import WORKLOADS
    return dict(WORKLOADS[name], name=name)


def make_inputs(w, miller):
    from paper_1305_7313_gb300 import synth
    from paper_1305_7313_gb300.workloads import cubic_cell
    cell = cubic_cell(w["L"])
    c = synth.orbitals(miller, cell, w["nb"], w["seed"])
    occ = np.full(w["nb"], 2.0)
    return cell, c, occ


class ClockSampler:
    """nvidia-smi SM clock / throttle samples while the timed region runs."""

    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.proc = None
        self.device_id = device_id

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device_id), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[4 + k].lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_id():
    """nvidia-smi's name for the current device: its UUID ("GPU-..."), else its index."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]


def time_form(plan, psi, occ, steps, warmup, want_dex=False, rank=0, world=1):
    """Warm up, then time `steps` applies between synchronised CUDA events."""
    import torch
    vpsi = torch.empty_like(psi)

    def step():
        if world == 1:
            plan.apply(psi, occ, vpsi, True, want_dex)
        else:  # band groups: this rank's shard of the pairs, then the sums over ranks
            from paper_1305_7313_gb300 import distributed
            distributed.apply(plan, psi, occ, vpsi_G=vpsi, want_dex=want_dex)

    for _ in range(warmup):
        step()
    plan.set_timing(True)
    phase_ms = {}
    launches = 0
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_id()) as clk:
        start.record()
        for _ in range(steps):
            step()
            st = plan.stats()
            launches += st["launches"]
            for k, v in st["phase_ms"].items():
                phase_ms[k] = phase_ms.get(k, 0.0) + v
        end.record()
        torch.cuda.synchronize()
    plan.set_timing(False)
    ms = start.elapsed_time(end)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=psi.device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return dict(ms=ms, phase_ms=phase_ms, launches=launches, stats=plan.stats(), clocks=clk.summary())


# DRAM bytes (read + write) per chain of the dominant kernel, from ncu captures
# of the 96^3 pair passes of the 64-band case at 38 chains per launch, one
# stream (profiles/pair_traffic_96.md); scaled
# to a launch by its chains, reported only for a captured band block (the
# orbital re-reads depend on it).
MEASURED_TRAFFIC_PER_CHAIN = {
    ("fp64", 96, "pair_inv", 8): 54.04e6, ("fp64", 96, "pair_inv", 16): 47.18e6, ("fp64", 96, "pair_inv", 32): 52.54e6,
    ("df64", 96, "pair_inv", 8): 57.45e6, ("df64", 96, "pair_inv", 16): 50.67e6, ("df64", 96, "pair_inv", 32): 53.20e6,
    ("mixed32", 96, "pair_inv", 8): 12.61e6, ("mixed32", 96, "pair_inv", 16): 19.28e6,
}


def pair_loop_ms(res, steps):
    """Device time per step of the pair passes (forward, column, inverse): the
    step time minus the phases around them, which run on the call's stream
    alone (the pair passes' launches may overlap on several streams)."""
    other = sum(res["phase_ms"].get(k, 0.0) for k in ("to_real", "to_sphere", "energy")) / steps
    return res["ms"] / steps - other


def pair_loop_rate(pairs, res, steps):
    """Pairs per second of the pair passes alone."""
    ms = pair_loop_ms(res, steps)
    return pairs / (ms * 1e-3) if ms > 0 else None


def measured_traffic(form, n, kernel, band_block, chains_per_launch):
    per = MEASURED_TRAFFIC_PER_CHAIN.get((form, n, kernel, band_block))
    if per is None:
        return None
    return per * chains_per_launch


def roofline(form, plan, res, steps, peaks, peak_src, band_block=16, streams=1):
    """Roofline of the dominant pair kernel (the phase with the largest device
    time), or of the three pair passes together when their launches overlap
    on several streams (a launch's duration then includes its neighbours')."""
    if streams > 1:
        return loop_roofline(form, plan, res, steps, peaks, peak_src, band_block, streams)
    n = plan.grid[0]
    ntot = float(n) ** 3
    nc = 2 * (n // 2 + 1)
    st = res["stats"]
    pair_phases = ["pair_fwd", "pair_col", "pair_inv"]
    dom = max(pair_phases, key=lambda k: res["phase_ms"].get(k, 0.0))
    launches = st["phase_launches"][dom] * steps
    ms_per_launch = res["phase_ms"][dom] / max(1, launches)
    chains_per_launch = st["chains"] / max(1, st["phase_launches"][dom])
    log2n = np.log2(n)
    if form in ("fp64", "df64"):
        # 5 n log2 n flops per complex line transform of length n; the plane passes
        # do 2 N^2 lines, the column pass N (N+2) lines forward and as many inverse
        per_chain = {"pair_fwd": 5 * ntot * 2 * log2n, "pair_inv": 5 * ntot * 2 * log2n,
                     "pair_col": 2 * 5 * ntot * log2n * nc / n}[dom]
        achieved = per_chain * chains_per_launch / (ms_per_launch * 1e-3) / 1e12
        mhz = res["clocks"].get("sm_mhz") or 2070.0
        per_clk = FP64_FLOPS_PER_CLK if form == "fp64" else DF64_FLOPS_PER_CLK
        peak = per_clk * 2070.0e6 / 1e12
        src = ("measured DFMA loop, 2070 MHz" if form == "fp64" else
               "measured FP32 FMA loop / 9.4 FP32 instructions per double-float flop, 2070 MHz")
        return {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": measured_traffic(form, n, dom, band_block, chains_per_launch),
                "peak_src": src, "frac_at_sampled_clock": achieved / (per_clk * mhz * 1e6 / 1e12),
                "ms_per_launch": ms_per_launch, "chains_per_launch": chains_per_launch}
    # Algorithmic bytes per chain (two pairs): the kept columns of the complex64
    # half spectrum (written by pair_fwd, read and written by pair_col, read by
    # pair_inv) plus the orbital and accumulator planes, each reused by the
    # chains of a band block: pair_fwd reads four orbital planes, pair_inv reads
    # four and read-modify-writes four accumulator planes.
    kept, total = plan.columns()
    hbytes = n * n * nc * 8.0 * kept / total
    plane = ntot * 4.0 / max(1, band_block)
    per_chain = {"pair_fwd": hbytes + 4 * plane, "pair_col": 2 * hbytes, "pair_inv": hbytes + 12 * plane}[dom]
    achieved = per_chain * chains_per_launch / (ms_per_launch * 1e-3) / 1e9
    peak = float(peaks["hbm_gbs"])
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": measured_traffic(form, n, dom, band_block, chains_per_launch),
            "peak_src": peak_src + " (hbm copy)", "bytes_per_chain": per_chain,
            "ms_per_launch": ms_per_launch, "chains_per_launch": chains_per_launch}


def golden_errors(plan, c, w):
    """Errors of `plan`'s apply on the first 64 bands of workload `w` against the
    oracle's stored values for the same 64 bands (E_x, dE_x/domega, V_x psi at
    sampled sphere positions; tests/golden/oracle_fullsize_N96_nb64.txt).  Run
    outside the timed region."""
    import importlib.util
    import torch
    spec = importlib.util.spec_from_file_location(
        "fullsize_record", os.path.join(ROOT, "tests", "golden", "fullsize_record.py"))
    rec_mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(rec_mod)
    case = rec_mod.CASE_OF_SEED.get(w["seed"])
    if case is None or plan.grid[0] != 96 or w["nb"] != rec_mod.NB_ALL or not os.path.exists(rec_mod.FILE):
        return None
    rec = rec_mod.load()
    sub = torch.from_numpy(np.ascontiguousarray(c[:rec_mod.NB])).cuda()
    vpsi, ex, dex = plan.apply(sub, np.full(rec_mod.NB, 2.0), want_dex=True)
    err = rec_mod.compare(rec, case, ex, dex, vpsi.cpu().numpy())
    err["against"] = "stored FP64 oracle, first 64 bands (E_x, dE/domega; V_x psi at %d sampled G)" % err.pop("samples")
    del sub, vpsi
    return err


def phase_share(res):
    """Shares of the three pair passes in their summed device time (rounded)."""
    ph = {k: res["phase_ms"].get("pair_" + k, 0.0) for k in ("fwd", "col", "inv")}
    tot = sum(ph.values())
    return {k: round(v / tot, 3) for k, v in ph.items()} if tot > 0 else None


def form_summary(res_line, roof, err):
    """The compact record of one form printed at the end of the JSON line."""
    out = {"workload": res_line["workload"], "value": res_line["value"], "unit": UNIT,
           "ms_per_step": res_line["ms_per_step"], "dtype": res_line["dtype"],
           "frac": roof["frac"], "bound": roof["bound"], "achieved": roof["achieved"],
           "peak": roof["peak"], "roof_unit": roof["unit"], "dominant": roof["kernel"],
           "traffic": roof["traffic"], "pair_loop_pairs_per_s": res_line["pair_loop_pairs_per_s"],
           "pass_share": res_line.get("pass_share"), "steps": res_line.get("steps")}
    if err:
        out.update({k: err[k] for k in ("max_abs_dVpsi_rel", "rel_dEx", "rel_ddEx_domega")})
    return out


def loop_roofline(form, plan, res, steps, peaks, peak_src, band_block, streams):
    """Achieved rate of the three pair passes together: their algorithmic flops
    (FP64, double-float) or bytes (mixed) per step over the pair loop's device
    time per step."""
    n = plan.grid[0]
    ntot = float(n) ** 3
    nc = 2 * (n // 2 + 1)
    chains = res["stats"]["chains"]
    ms = pair_loop_ms(res, steps)
    label = "pair passes (fwd + col + inv, launches on %d streams)" % streams
    if form in ("fp64", "df64"):
        log2n = np.log2(n)
        per_chain = 5 * ntot * 2 * log2n * 2 + 2 * 5 * ntot * log2n * nc / n
        achieved = per_chain * chains / (ms * 1e-3) / 1e12
        per_clk = FP64_FLOPS_PER_CLK if form == "fp64" else DF64_FLOPS_PER_CLK
        peak = per_clk * 2070.0e6 / 1e12
        mhz = res["clocks"].get("sm_mhz") or 2070.0
        src = ("measured DFMA loop, 2070 MHz" if form == "fp64" else
               "measured FP32 FMA loop / 9.4 FP32 instructions per double-float flop, 2070 MHz")
        out = {"bound": "alu", "kernel": label, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
               "frac": achieved / peak, "peak_src": src,
               "frac_at_sampled_clock": achieved / (per_clk * mhz * 1e6 / 1e12)}
    else:
        kept, total = plan.columns()
        hbytes = n * n * nc * 8.0 * kept / total
        plane = ntot * 4.0 / max(1, band_block)
        per_chain = 4 * hbytes + 16 * plane
        achieved = per_chain * chains / (ms * 1e-3) / 1e9
        peak = float(peaks["hbm_gbs"])
        out = {"bound": "hbm", "kernel": label, "achieved": achieved, "peak": peak, "unit": "GB/s",
               "frac": achieved / peak, "peak_src": peak_src + " (hbm copy)", "bytes_per_chain": per_chain}
    per = MEASURED_LOOP_TRAFFIC_PER_CHAIN.get((form, n, band_block))
    out.update({"traffic": per * chains if per else None, "traffic_unit": "DRAM bytes per step (ncu, all three kernels)",
                "ms_pair_loop": ms, "chains_per_step": chains})
    return out


# DRAM bytes (read + write) per chain of the three pair kernels together, from
# ncu captures of the 96^3 pair passes on one stream at 38 chains per launch
# (profiles/pair_traffic_96.md), by form and band block; scaled to a step by
# its chains.  The mixed form's column pass has changed since its capture
# (CTAs of 56 lines), so its loop has no measured figure
MEASURED_LOOP_TRAFFIC_PER_CHAIN = {
    ("fp64", 96, 8): 95.61e6, ("fp64", 96, 16): 86.80e6, ("fp64", 96, 32): 94.01e6,
    ("df64", 96, 8): 98.40e6, ("df64", 96, 16): 90.15e6, ("df64", 96, 32): 94.48e6,
}


def fixed_blocks(plan, args):
    """--chain-batch / --band-block given: set them and report them as the choice."""
    if args.chain_batch:
        plan.set_batch(args.chain_batch)
    if args.band_block:
        plan.set_band_block(args.band_block)
    if args.tiles:
        plan.set_tiling([int(x) for x in args.tiles])
    plan.set_streams(args.streams)
    return {"chain_batch": args.chain_batch, "band_block": args.band_block or 16, "tiles": args.tiles,
            "streams": args.streams, "tuned_on_bands": 0, "candidates": 0}


def tune_on_subset(plan, c, occ, nbands, reps=2):
    """Pick chain_batch / band_block for `plan` on its first `nbands` orbitals."""
    import torch
    from paper_1305_7313_gb300.autotune import tune_apply
    sub = torch.from_numpy(np.ascontiguousarray(c[:nbands])).cuda()
    res = tune_apply(plan, sub, occ[:nbands], reps=reps, use_cache=False)
    del sub
    return {"chain_batch": res["chain_batch"], "band_block": res["band_block"], "streams": res.get("streams", 1),
            "tiles": res.get("tiles"),
            "tiling": tiling_text(res.get("tiling")), "tuned_on_bands": nbands, "candidates": len(res["table"])}


def tiling_text(tiling):
    """'fwd 12x4x2/8 col 12x8/4 inv 12x8/4': radix plan / threads per line per pair pass."""
    if not tiling:
        return None
    short = {"pair_fwd": "fwd", "pair_col": "col", "pair_inv": "inv"}
    return " ".join("%s %s/%d" % (short[k], "x".join(str(r) for r in v["radices"]), v["threads_per_line"])
                    for k, v in tiling.items())


def run_batched(args, peaks, peak_src):
    """16 uneven systems (grids 48/64/72/96, 32-384 bands) in one persistent launch."""
    import torch
    from paper_1305_7313_gb300 import FockBatch, FockPlan
    from paper_1305_7313_gb300.autotune import tune_batch
    from paper_1305_7313_gb300.workloads import batched_systems, cubic_cell
    systems = batched_systems()
    if args.nb:
        for sy in systems:
            sy["nb"] = min(sy["nb"], args.nb)
    plans, psis, occs = [], [], []
    for sy in systems:
        p = FockPlan(sy["N"], cubic_cell(sy["L"]), sy["ecut"], sy["kernel"], sy["omega"], sy["prec"])
        _, c, occ = make_inputs(sy, p.miller)
        plans.append(p)
        psis.append(torch.from_numpy(c).cuda())
        occs.append(occ)
    pairs = sum(sy["nb"] * (sy["nb"] + 1) // 2 for sy in systems)
    tuned = {"options": {"persistent": args.batch_mode}, "band_block": 16}
    if not args.no_tune:
        tuned = tune_batch(plans, psis, occs, slot_chains=(4, 8, 16), rings=(3,), ctas_per_sm=(0,),
                           persistent=(1, 2, 0), reps=1, use_cache=False)
    batch = FockBatch(plans, psis, occs, **tuned["options"])
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    pms = []
    with ClockSampler(gpu_id()) as clk:
        start.record()
        for _ in range(args.steps):
            batch.run()
            pms.append(batch.info()["persist_ms"])
        end.record()
        torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    info = batch.info()
    # algorithmic bytes of the pair passes, per chain of each system: the kept
    # columns of the complex64 half spectrum are written (fwd), read and
    # written (col) and read (inv); the forward pass reads four orbital planes
    # and the inverse pass reads four and read-modify-writes four accumulator
    # planes, each counted once per band block
    bb = tuned.get("band_block", 16)
    nbytes = 0.0
    for sy, p in zip(systems, plans):
        n = sy["N"]
        kept, total = p.columns()
        chains = (sy["nb"] * (sy["nb"] + 1) // 2 + 1) // 2
        hbytes = n * n * 2 * (n // 2 + 1) * 8.0 * kept / total
        nbytes += chains * (4 * hbytes + 16 * n ** 3 * 4.0 / max(1, min(bb, sy["nb"])))
    pm = statistics.median(pms)
    achieved = nbytes / (pm * 1e-3) / 1e9
    batch.close()
    for p in plans:
        p.close()
    mode = int(tuned["options"].get("persistent", 1))
    traffic = None
    if args.nb is None and bb == BATCH_DRAM_BAND_BLOCK and mode == 0:
        # DRAM bytes per chain of the pair passes (ncu, 64-band systems), scaled by chains
        traffic = sum(((sy["nb"] * (sy["nb"] + 1) // 2 + 1) // 2) * BATCH_DRAM_PER_CHAIN.get(sy["N"], float("nan"))
                      for sy in systems)
        traffic = None if traffic != traffic else traffic
    nbytes_kernel = {0: "pair passes (graph branches)", 1: "k_pair_persistent", 2: "k_pair_dataflow"}[mode]
    persistent = mode != 0
    return {"workload": "batched16_mixed32_sa_N48-96_L13.5-27",
            "mode": {0: "graph branches of size-specialised launches", 1: "persistent launch",
                     2: "dataflow launch (one CTA per task)"}[mode],
            "value": pairs * args.steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "pairs": pairs, "dtype": "f32", "graph": True, "persistent_launches_per_step": 1 if persistent else 0,
            "gpu_launches_per_step": info["launches"], "persistent_grid": info["grid"],
            "segments": info["segments"], "tasks": info["tasks"],
            "roofline": {"bound": "hbm", "kernel": nbytes_kernel, "achieved": achieved,
                         "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                         "frac": achieved / float(peaks["hbm_gbs"]), "traffic": traffic,
                         "algorithmic_bytes": nbytes, "peak_src": peak_src + " (hbm copy)", "ms_pair_passes": pm},
            "tuned": {"options": tuned["options"], "band_block": tuned["band_block"],
                      "best_ms_by_mode": best_by_mode(tuned.get("table", []))},
            "clocks": clk.summary()}


# DRAM bytes (read + write) per chain of the three pair passes of the batch's
# systems, by grid size, at band block 16: an ncu capture of every pair launch
# of the 64-band version of the batch as graph branches (launches serialised
# by ncu; profiles/pair_traffic_96.md).  The 96^3 systems' column pass has
# changed since (CTAs of 56 lines), so the batch has no measured total
BATCH_DRAM_PER_CHAIN = {48: 3.077e6, 64: 7.361e6, 72: 10.790e6}
BATCH_DRAM_BAND_BLOCK = 16


def best_by_mode(table):
    """Fastest tuner candidate per pair-pass mode (persistent launch vs graph branches)."""
    out = {}
    for r in table:
        key = {0: "branches", 1: "persistent", 2: "dataflow"}[int(r["options"].get("persistent", 1))]
        if key not in out or r["ms"] < out[key]:
            out[key] = r["ms"]
    return out


def run_kpoints(args, peaks, peak_src):
    """2x2x2 Monkhorst-Pack mesh (k in {0, 1/2}^3, weights 1/8), 48^3 grid,
    L = 13.5 bohr, Ecut = 12 Ha, 32 bands per k, erfc kernel, mixed form."""
    import itertools
    import torch
    from paper_1305_7313_gb300 import FockKPlan, PREC_MIXED32, synth
    from paper_1305_7313_gb300.workloads import ERFC, cubic_cell
    n, L, ecut, nb, omega = 48, 13.5, 12.0, 32, 0.106
    if args.nb:
        nb = min(nb, args.nb)
    kpts = np.array(list(itertools.product([0.0, 0.5], repeat=3)))
    wk = np.full(len(kpts), 1.0 / len(kpts))
    cell = cubic_cell(L)
    plan = FockKPlan(n, cell, ecut, kpts, wk, ERFC, omega, PREC_MIXED32)
    psi = [torch.from_numpy(synth.orbitals_k(plan.miller(k), cell, kpts[k], nb, 2300 + k)).cuda()
           for k in range(len(kpts))]
    occ = np.full((len(kpts), nb), 2.0)
    for _ in range(args.warmup):
        plan.apply(psi, occ)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(args.steps):
        plan.apply(psi, occ)
    end.record()
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    ns = len(kpts) * nb
    pairs = ns * (ns + 1) // 2
    nbytes = pairs * 4.0 * n**3 * 8.0  # complex64 full spectrum: written, read + written, read
    achieved = nbytes * args.steps / (ms * 1e-3) / 1e9
    # DRAM bytes (read + write) per pair of the three k-point pair kernels, from
    # an ncu capture of every pair launch of this leg (profiles/kpair_traffic_48.md)
    traffic = KPOINT_DRAM_PER_PAIR * pairs if nb == 32 else None
    plan.close()
    return {"workload": "kpoints8_mixed32_erfc_L13.5_N48_nb32", "kpoints": len(kpts), "bands_per_k": nb,
            "value": pairs * args.steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "pairs": pairs, "dtype": "f32",
            "roofline": {"bound": "hbm", "kernel": "pair passes (whole step)", "achieved": achieved,
                         "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                         "frac": achieved / float(peaks["hbm_gbs"]), "traffic": traffic,
                         "traffic_unit": "DRAM bytes per step (ncu, all three kernels)",
                         "peak_src": peak_src + " (hbm copy)"}}


KPOINT_DRAM_PER_PAIR = 3.351e6


def run_fixed(args):
    """The exchange operator fixed by an occupied set and applied to trial
    orbitals, as in an SCF inner loop: 96^3, L = 27 bohr, Ecut = 12 Ha, erfc
    kernel (omega 0.106), mixed form; 256 occupied and 256 trial orbitals,
    V_x fixed once outside the timed region, each step one apply to the trial
    set (256 x 256 pairs)."""
    import torch
    from paper_1305_7313_gb300 import FockPlan, synth
    w = workload("gamma_mixed32_erfc_L27_N96_nb512")
    nocc = ntrial = 256
    if args.nb:
        nocc = ntrial = min(nocc, args.nb)
    from paper_1305_7313_gb300.workloads import cubic_cell
    cell = cubic_cell(w["L"])
    plan = FockPlan(w["N"], cell, w["ecut"], w["kernel"], w["omega"], w["prec"])
    psi = torch.from_numpy(synth.orbitals(plan.miller, cell, nocc, w["seed"])).cuda()
    phi = torch.from_numpy(synth.orbitals(plan.miller, cell, ntrial, w["seed"] + 1000)).cuda()
    plan.set_occupied(psi, np.full(nocc, 2.0))
    out = torch.empty_like(phi)
    for _ in range(args.warmup):
        plan.apply_fixed(phi, out)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(args.steps):
        plan.apply_fixed(phi, out)
    end.record()
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    plan.close()
    pairs = nocc * ntrial
    return {"workload": "fixed_mixed32_erfc_L27_N96_nocc256_ntrial256", "value": pairs * args.steps / (ms * 1e-3),
            "unit": UNIT, "ms_per_step": ms / args.steps, "pairs": pairs, "dtype": "f32"}


def run_sternheimer(args):
    """Sternheimer linear response by CG with band regrouping (FP64): 48^3
    grid, L = 13.5 bohr, Ecut = 12 Ha, H = kinetic + a model local potential
    (three Gaussian wells), 32 occupied kets and 32 right-hand kets (seeded
    orthonormal sets, the right-hand ones scaled by 1, 1e-2, 1e-4, 1e-6 in
    turn), eps_n below the spectrum of H (every system positive definite),
    alpha = 1, residual threshold 1e-8.  Each step is one solve
    (the per-iteration readback of the residual norms included)."""
    import torch
    from paper_1305_7313_gb300 import FockPlan, PREC_FP64, synth
    from paper_1305_7313_gb300.workloads import SPENCER_ALAVI, cubic_cell
    n, L, ecut, nocc, nrhs = 48, 13.5, 12.0, 32, 32
    if args.nb:
        nocc, nrhs = min(nocc, args.nb), min(nrhs, args.nb)
    cell = cubic_cell(L)
    plan = FockPlan(n, cell, ecut, SPENCER_ALAVI, None, PREC_FP64)
    v = synth.model_potential((n, n, n), cell, 11)
    u = torch.from_numpy(synth.orbitals(plan.miller, cell, nocc, 2400)).cuda()
    # right-hand kets of norms 1, 1e-2, 1e-4, 1e-6 in turn: the bands converge
    # after different numbers of updates, so the regrouping shrinks the set
    scale = 10.0 ** (-2 * (np.arange(nrhs) % 4))
    wk = torch.from_numpy(synth.orbitals(plan.miller, cell, nrhs, 2401) * scale[:, None]).cuda()
    vd = torch.from_numpy(np.ascontiguousarray(v)).cuda()
    eps = v.min() - 1.0 - 0.01 * np.arange(nrhs)
    tol = 1e-8
    for _ in range(max(1, args.warmup)):
        plan.sternheimer(vd, u, eps, wk, 1.0, tol)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    updates = 0
    start.record()
    for _ in range(args.steps):
        _, iters, res = plan.sternheimer(vd, u, eps, wk, 1.0, tol)
        updates += int(np.sum(iters))
    end.record()
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    plan.close()
    return {"workload": "sternheimer_fp64_N48_L13.5_nocc32_nrhs32", "value": updates / (ms * 1e-3),
            "unit": "band CG updates/s", "ms_per_step": ms / args.steps, "npw": int(plan.npw),
            "iterations_max": int(np.max(iters)), "iterations_min": int(np.min(iters)),
            "iterations_mean": float(np.mean(iters)),
            "residual_max": float(np.max(res)), "dtype": "f64"}


def run_cufft_comparison(args, w, nbands=128, chunk=32):
    """The same apply written with cuFFT (torch.fft) and torch element-wise ops,
    timed on the first `nbands` bands of workload `w` in FP64 and in complex64:
    a comparison line, not part of the library.  Real pair densities go through
    R2C/C2R transforms; pairs (i, j >= i) are taken `chunk` at a time."""
    import torch
    from paper_1305_7313_gb300 import FockPlan, PREC_FP64
    from paper_1305_7313_gb300.workloads import cubic_cell
    n, L = w["N"], w["L"]
    nb = min(nbands, w["nb"])
    plan = FockPlan(n, cubic_cell(L), w["ecut"], w["kernel"], w["omega"], PREC_FP64)
    cell, c, occ = make_inputs(dict(w, nb=w["nb"]), plan.miller)
    c, occ = np.ascontiguousarray(c[:nb]), occ[:nb]
    psi_dev = torch.from_numpy(c).cuda()
    _, ex_fock, _ = plan.apply(psi_dev, occ, want_ex=True)
    mill = plan.miller
    plan.close()
    vol = L ** 3
    b = 2.0 * np.pi / L
    m = np.fft.fftfreq(n, 1.0 / n)
    mh = np.arange(n // 2 + 1)
    g2 = b * b * (m[:, None, None] ** 2 + m[None, :, None] ** 2 + mh[None, None, :] ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        if w["kernel"] == 0:
            rc = (3.0 * vol / (4.0 * np.pi)) ** (1.0 / 3.0)
            v = 8.0 * np.pi * np.sin(0.5 * np.sqrt(g2) * rc) ** 2 / g2
            v[0, 0, 0] = 2.0 * np.pi * rc * rc
        else:
            om = w["omega"]
            v = -4.0 * np.pi * np.expm1(-g2 / (4.0 * om * om)) / g2
            v[0, 0, 0] = np.pi / (om * om)
    wk3 = np.full(n // 2 + 1, 2.0)
    wk3[0] = 1.0
    if n % 2 == 0:
        wk3[-1] = 1.0
    flat = ((mill[:, 0] % n) * n + (mill[:, 1] % n)) * n + (mill[:, 2] % n)
    idx = torch.from_numpy(flat.astype(np.int64)).cuda()
    out = {}
    for name, rdt, cdt in (("fp64", torch.float64, torch.complex128), ("mixed32", torch.float32, torch.complex64)):
        vt = torch.from_numpy(v).to("cuda", rdt)
        wt = torch.from_numpy(wk3).to("cuda", torch.float64)
        f = torch.from_numpy(occ).to("cuda", rdt)
        cg = psi_dev.to(cdt)

        def apply():
            x = torch.zeros(nb, n ** 3, dtype=cdt, device="cuda")
            x[:, idx] = cg
            psi = torch.fft.ifftn(x.view(nb, n, n, n), dim=(1, 2, 3)).real * (n ** 3 / vol ** 0.5)
            wacc = torch.zeros_like(psi)
            ex = torch.zeros((), dtype=torch.float64, device="cuda")
            for i in range(nb):
                for j0 in range(i, nb, chunk):
                    j1 = min(nb, j0 + chunk)
                    rho = psi[i] * psi[j0:j1]
                    fr = torch.fft.rfftn(rho, dim=(1, 2, 3))
                    e = ((fr.real.double() ** 2 + fr.imag.double() ** 2) * vt.double() * wt).sum(dim=(1, 2, 3))
                    fj = f[j0:j1].double()
                    mult = torch.full_like(fj, 2.0)
                    if j0 == i:
                        mult[0] = 1.0
                    ex = ex + (-(vol / 2.0) / float(n) ** 6) * float(occ[i]) * (mult * fj * e).sum()
                    phi = torch.fft.irfftn(fr * vt, s=(n, n, n), dim=(1, 2, 3))
                    wacc[j0:j1] -= f[i] * psi[i] * phi
                    s = (f[j0:j1, None, None, None] * psi[j0:j1] * phi)
                    if j0 == i:
                        s = s[1:]
                    wacc[i] -= s.sum(0)
            y = torch.fft.fftn(wacc, dim=(1, 2, 3)).reshape(nb, -1)[:, idx] * (vol ** 0.5 / n ** 3)
            return y, ex

        y, ex = apply()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        reps = 2
        for _ in range(reps):
            y, ex = apply()
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / reps
        pairs = nb * (nb + 1) // 2
        out[name] = {"value": pairs / (ms * 1e-3), "unit": UNIT, "ms_per_apply": ms,
                     "rel_dEx_vs_fock_fp64": abs(float(ex) - ex_fock) / abs(ex_fock)}
        del y, cg
        torch.cuda.empty_cache()
    out["sample"] = "first %d bands (%d pairs), torch.fft R2C/C2R" % (nb, nb * (nb + 1) // 2)
    return out


def run_autograd(args):
    """E_x(psi, omega) forward + backward through the torch.autograd.Function:
    72^3 grid, L = 20 bohr, Ecut = 12 Ha, 256 bands, erfc kernel (omega = 0.106),
    complex64 orbitals, mixed form; gradients w.r.t. psi and omega."""
    import torch
    from paper_1305_7313_gb300 import FockPlan, synth
    from paper_1305_7313_gb300.autograd import exchange_energy
    w = workload("grad_erfc_L20_N72_nb256")
    if args.nb:
        w["nb"] = min(w["nb"], args.nb)
    n = w["N"]
    from paper_1305_7313_gb300.workloads import cubic_cell
    cell = cubic_cell(w["L"])
    with FockPlan(n, cell, w["ecut"], w["kernel"], w["omega"], w["prec"]) as probe:
        mill = probe.miller
    c = synth.orbitals(mill, cell, w["nb"], w["seed"])
    occ = np.full(w["nb"], 2.0)
    psi = torch.from_numpy(c).to("cuda", torch.complex64).requires_grad_(True)
    omega = torch.tensor(w["omega"], dtype=torch.float64, requires_grad=True)

    def step():
        psi.grad = None
        omega.grad = None
        e = exchange_energy(psi, occ, n, cell, w["ecut"], w["kernel"], omega, w["prec"])
        e.backward()
        return e

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        e = step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    pairs = w["nb"] * (w["nb"] + 1) // 2
    return {"workload": w["name"], "value": pairs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "pairs": pairs, "dtype": "f32 (complex64 orbitals and gradients, FP64 energy sums)",
            "e_x": float(e.detach()), "de_domega": float(omega.grad), "grad_psi_norm": float(psi.grad.abs().max())}


def cpu_baseline(w, nbands_sample=32):
    """The FP64 oracle on the first `nbands_sample` bands of the workload."""
    import oracle
    from paper_1305_7313_gb300 import synth
    from paper_1305_7313_gb300.workloads import cubic_cell
    n = w["N"]
    cell = cubic_cell(w["L"])
    mill, _ = oracle.gsphere((n, n, n), cell, w["ecut"])
    c = synth.orbitals(mill, cell, w["nb"], w["seed"])[:nbands_sample]
    occ = np.full(nbands_sample, 2.0)
    kind = "spencer_alavi" if w["kernel"] == 0 else "erfc"
    t0 = time.perf_counter()
    oracle.fock_apply(c, occ, mill, (n, n, n), cell, kind, w["omega"])
    dt = time.perf_counter() - t0
    pairs = nbands_sample * (nbands_sample + 1) // 2
    return {"value": pairs / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle fock_apply (V_x psi and E_x) of the first %d bands of the %s workload "
                      "(%d unique pairs, %.1f s)" % (nbands_sample, w["name"], pairs, dt),
            "seconds": dt}


def run_reference(args, rank):
    if rank != 0:
        return
    w = workload("gamma_fp64_L27_N96_nb512")
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(cpu_baseline(w, args.ref_bands))
    timed = vals[args.warmup:]
    v = statistics.median(x["value"] for x in timed)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(x["seconds"] for x in timed),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w["name"], "grid": 96, "L_bohr": 27.0, "ecut_ha": 12.0,
                       "nbands": 512, "pairs": 131328},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": timed[0]["cores"], "kind": "oracle",
                             "sample": timed[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fock", choices=["fock", "reference"])
    ap.add_argument("--workload", default="gamma_fp64_L27_N96_nb512")
    ap.add_argument("--mixed-workload", default="gamma_mixed32_erfc_L27_N96_nb512")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--df64-workload", default="gamma_df64_L27_N96_nb512")
    ap.add_argument("--no-df64", action="store_true", help="skip the double-float form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-bands", type=int, default=32)
    ap.add_argument("--nb", type=int, default=None,
                    help="override the band count of the workloads (small profiling cases)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-kpoints", action="store_true")
    ap.add_argument("--no-autograd", action="store_true", help="skip the E_x(psi, omega) autograd leg")
    ap.add_argument("--no-fixed", action="store_true", help="skip the fixed-operator (trial orbitals) leg")
    ap.add_argument("--no-sternheimer", action="store_true", help="skip the Sternheimer CG leg")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--chain-batch", type=int, default=0,
                    help="with --no-tune: chains per pair-pass launch of the Gamma-point forms")
    ap.add_argument("--band-block", type=int, default=0,
                    help="with --no-tune: band block of the Gamma-point pair schedule")
    ap.add_argument("--streams", type=int, default=1,
                    help="with --no-tune: streams the pair-pass launches rotate over (1-4)")
    ap.add_argument("--tiles", default="",
                    help="with --no-tune: FFT tiling of the forward, column and inverse passes, e.g. 100")
    ap.add_argument("--batch-mode", type=int, default=0, choices=[0, 1, 2],
                    help="with --no-tune: pair passes of the batch as graph branches (0), one persistent "
                         "launch (1) or one dataflow launch (2)")
    ap.add_argument("--side-steps", type=int, default=5,
                    help="timed steps of the end-to-end and double-float legs (at most --steps): each "
                         "of their steps takes seconds at 96^3/512 bands")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparison line")
    ap.add_argument("--cufft-bands", type=int, default=128)
    ap.add_argument("--tune-bands", type=int, default=64,
                    help="band count of the subset the apply's pair-block parameters are tuned on")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1305_7313_gb300 import FockPlan, PREC_FP64, PREC_MIXED32
    peaks, peak_src = load_peaks()

    # ---- FP64 form (the headline workload)
    w = workload(args.workload)
    if args.nb:
        w["nb"] = args.nb
    n = w["N"]
    from paper_1305_7313_gb300.workloads import cubic_cell
    plan = FockPlan(n, cubic_cell(w["L"]), w["ecut"], w["kernel"], w["omega"], w["prec"])
    cell, c, occ = make_inputs(w, plan.miller)
    tuned = None
    if not args.no_tune:
        tuned = tune_on_subset(plan, c, occ, min(w["nb"], max(8, args.tune_bands // 2)), reps=1)
    elif args.chain_batch or args.band_block or args.tiles or args.streams > 1:
        tuned = fixed_blocks(plan, args)
    psi = torch.from_numpy(c).cuda()
    pairs = w["nb"] * (w["nb"] + 1) // 2
    res = time_form(plan, psi, occ, args.steps, args.warmup, rank=rank, world=world)
    ms_step = res["ms"] / args.steps
    value = pairs * args.steps / (res["ms"] * 1e-3)
    form = {PREC_FP64: "fp64", PREC_MIXED32: "mixed32"}.get(w["prec"], "df64")
    roof = roofline(form, plan, res, args.steps, peaks, peak_src, tuned["band_block"] if tuned else 16,
                    tuned.get("streams", 1) if tuned else 1)
    err = golden_errors(plan, c, w) if world == 1 else None

    # ---- end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e and world == 1:
        host = torch.from_numpy(c).pin_memory()
        out = torch.empty(host.shape, dtype=host.dtype, pin_memory=True)
        plan.apply_host(host, occ, out)
        torch.cuda.synchronize()
        k_e2e = min(args.steps, args.side_steps)  # each step repeats the headline's (seconds at 96^3/512)
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            plan.apply_host(host, occ, out)
        dt = time.perf_counter() - t0
        nbytes = host.numel() * host.element_size()
        e2e = {"value": pairs * k_e2e / dt, "unit": UNIT, "h2d_bytes_per_step": nbytes + 8 * w["nb"],
               "d2h_bytes_per_step": nbytes + 16, "ms_per_step": 1e3 * dt / k_e2e, "steps": k_e2e}
        del host, out
    del psi
    plan.close()
    torch.cuda.empty_cache()

    # ---- mixed form, same 96^3 / 512-band shape
    mixed = None
    if not args.no_mixed:
        wm = workload(args.mixed_workload)
        if args.nb:
            wm["nb"] = args.nb
        planm = FockPlan(wm["N"], cubic_cell(wm["L"]), wm["ecut"], wm["kernel"], wm["omega"], wm["prec"])
        _, cm, occm = make_inputs(wm, planm.miller)
        tunedm = None
        if not args.no_tune:
            tunedm = tune_on_subset(planm, cm, occm, min(wm["nb"], args.tune_bands))
        elif args.chain_batch or args.band_block or args.tiles or args.streams > 1:
            tunedm = fixed_blocks(planm, args)
        psim = torch.from_numpy(cm).cuda()
        resm = time_form(planm, psim, occm, args.steps, args.warmup, rank=rank, world=world)
        pm = wm["nb"] * (wm["nb"] + 1) // 2
        mixed = {"workload": wm["name"], "value": pm * args.steps / (resm["ms"] * 1e-3), "unit": UNIT,
                 "steps": args.steps,
                 "ms_per_step": resm["ms"] / args.steps, "dtype": "f32",
                 "roofline": roofline("mixed32", planm, resm, args.steps, peaks, peak_src,
                                      tunedm["band_block"] if tunedm else 16, tunedm.get("streams", 1) if tunedm else 1),
                 "pair_loop_pairs_per_s": pair_loop_rate(pm, resm, args.steps), "pass_share": phase_share(resm),
                 "gpu_launches": resm["launches"], "clocks": resm["clocks"], "tuned": tunedm}
        mixed["summary"] = form_summary(mixed, mixed["roofline"], golden_errors(planm, cm, wm) if world == 1 else None)
        planm.close()
        del psim
        torch.cuda.empty_cache()

    # ---- double-float form of the FP64 workload (FP64-class accuracy, FP32 pipe)
    df = None
    if not args.no_df64:
        wd = workload(args.df64_workload)
        if args.nb:
            wd["nb"] = args.nb
        pland = FockPlan(wd["N"], cubic_cell(wd["L"]), wd["ecut"], wd["kernel"], wd["omega"], wd["prec"])
        _, cd, occd = make_inputs(wd, pland.miller)
        tunedd = None
        if not args.no_tune:
            tunedd = tune_on_subset(pland, cd, occd, min(wd["nb"], args.tune_bands), reps=1)
        elif args.chain_batch or args.band_block or args.tiles or args.streams > 1:
            tunedd = fixed_blocks(pland, args)
        psid = torch.from_numpy(cd).cuda()
        kd = min(args.steps, args.side_steps)
        resd = time_form(pland, psid, occd, kd, args.warmup, rank=rank, world=world)
        pd = wd["nb"] * (wd["nb"] + 1) // 2
        df = {"workload": wd["name"], "value": pd * kd / (resd["ms"] * 1e-3), "unit": UNIT, "steps": kd,
              "ms_per_step": resd["ms"] / kd, "dtype": "f32x2 (double-float)",
              "roofline": roofline("df64", pland, resd, kd, peaks, peak_src,
                                   tunedd["band_block"] if tunedd else 16, tunedd.get("streams", 1) if tunedd else 1),
              "pair_loop_pairs_per_s": pair_loop_rate(pd, resd, kd), "pass_share": phase_share(resd),
              "gpu_launches": resd["launches"], "clocks": resd["clocks"], "tuned": tunedd}
        df["summary"] = form_summary(df, df["roofline"], golden_errors(pland, cd, wd) if world == 1 else None)
        pland.close()
        del psid
        torch.cuda.empty_cache()

    batched = None
    if not args.no_batched and world == 1:
        batched = run_batched(args, peaks, peak_src)
        torch.cuda.empty_cache()

    kpoints = None
    if not args.no_kpoints and world == 1:
        kpoints = run_kpoints(args, peaks, peak_src)
        torch.cuda.empty_cache()

    autograd = None
    if not args.no_autograd and world == 1:
        autograd = run_autograd(args)
        torch.cuda.empty_cache()

    fixed = None
    if not args.no_fixed and world == 1:
        fixed = run_fixed(args)
        torch.cuda.empty_cache()

    stern = None
    if not args.no_sternheimer and world == 1:
        stern = run_sternheimer(args)
        torch.cuda.empty_cache()

    cufft = None
    if not args.no_cufft and world == 1:
        cufft = run_cufft_comparison(args, w, args.cufft_bands)
        torch.cuda.empty_cache()

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w, args.ref_bands)
        cpu.pop("seconds", None)
    def brief_tuned(t):
        return None if t is None else {k: t.get(k) for k in ("chain_batch", "band_block", "streams", "tiling")}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": {"fp64": "f64", "mixed32": "f32", "df64": "f32x2 (double-float)"}[form],
        "data": "synthetic",
        "config": {"workload": w["name"], "grid": n, "L_bohr": w["L"], "ecut_ha": w["ecut"],
                   "nbands": w["nb"], "pairs": pairs, "npw": plan.npw,
                   "kernel": "spencer_alavi" if w["kernel"] == 0 else "erfc",
                   "l2": "inputs larger than L2 (real-space orbitals and accumulators %.1f GB each)"
                         % (w["nb"] * n**3 * (4 if form == "mixed32" else 8) / 1e9),
                   "parallelism": "band-group shards + all-reduce" if world > 1 else "single GPU"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
        "errors": err,
        "pair_loop_pairs_per_s": pair_loop_rate(pairs, res, args.steps),
        "pass_share": phase_share(res),
        "tuned": brief_tuned(tuned),
        "batched": batched,
        "kpoints": kpoints,
        "autograd": autograd,
        "fixed_operator": fixed,
        "sternheimer": stern,
        "cufft_comparison": cufft,
        # the two other forms of the metric last, compact
        "df64_summary": dict(df["summary"], tuned=brief_tuned(df["tuned"])) if df else None,
        "mixed32_summary": dict(mixed["summary"], tuned=brief_tuned(mixed["tuned"])) if mixed else None,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
