"""Autotuner for the pair-block parameters of the apply and of the batched form.

The knobs are the ones that decide how pair work maps onto the GPU:

* ``chain_batch`` — band-pair chains (two pairs per complex transform) per
  launch of the pair passes, i.e. the size of the transform buffer a launch
  streams through L2/HBM;
* ``band_block`` — bands per block of the pair schedule (pairs are visited in
  band_block x band_block blocks, so consecutive chains share orbitals and
  accumulators in L2);
* ``streams`` — how many streams the launches of the pair passes rotate over
  (neighbouring launches overlap on the GPU);
* ``tiling`` — the FFT tiling (radix plan and threads per line) of each of the
  three pair passes, where the library compiled two (``FockPlan.tilings()``);
  searched one pass at a time after the pair-block search;
* for batches: ``persistent`` (1: one persistent launch for all systems; 2:
  one dataflow launch with a CTA per task; 0: size-specialised launches on
  one graph branch per system), ``slot_chains``
  (chains of the largest grid per transform-buffer slot of the persistent
  launch), ``ring`` (slots in flight) and ``ctas_per_sm`` (resident CTAs per
  SM of the persistent launch).

Each candidate is timed on the caller's own inputs with CUDA events (one
warm-up, then the median of ``reps`` runs) and the fastest is returned.  Results
are cached in a JSON file keyed by the workload's shape (``FOCK_TUNE_CACHE``,
default ``~/.cache/fockx/tune.json``) so a second process skips the search.
"""

import itertools
import json
import os
import statistics

from .plan import FockBatch


def _cache_path():
    return os.environ.get("FOCK_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "fockx",
                                                          "tune.json"))


def _load_cache():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(key, value):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        data = _load_cache()
        data[key] = value
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _time_ms(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    out = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
    return statistics.median(out)


PASSES = ("pair_fwd", "pair_col", "pair_inv")


def tune_apply(plan, psi, occ, chain_batches=(8, 17, 19, 32, 38), band_blocks=(8, 16, 32), reps=2,
               use_cache=True, tiling=True, streams=(2, 3, 4)):
    """Fastest (chain_batch, band_block), stream count and FFT tiling for
    ``plan.apply(psi, occ)``; sets them on the plan.

    The pair-block grid is timed on one stream at the default tiling; then
    each stream count of ``streams`` with the best chain batch and with twice
    it (launches on several streams overlap, and larger ones fill the GPU
    better side by side); then, one pair pass at a time, the pass's other
    tiling is timed at the best setting so far and kept if faster.  Returns
    ``{"chain_batch", "band_block", "streams", "tiles", "tiling", "ms",
    "table"}``; ``tiling`` names each pass's chosen radix plan and threads per
    line.
    """
    key = "apply|%s|N%d|prec%d|nb%d" % (_gpu_name(), plan.grid[0], plan.precision, psi.shape[0])
    has_tiling = tiling and hasattr(plan, "tilings")
    has_streams = bool(streams) and hasattr(plan, "set_streams")
    if use_cache:
        hit = _load_cache().get(key)
        if hit and ("tiles" in hit or not has_tiling) and ("streams" in hit or not has_streams):
            plan.set_batch(hit["chain_batch"])
            plan.set_band_block(hit["band_block"])
            if has_tiling:
                plan.set_tiling(hit["tiles"])
            if has_streams:
                plan.set_streams(hit["streams"])
            return dict(hit, cached=True)
    table = []
    tiles = [0, 0, 0]
    if has_tiling:
        plan.set_tiling(tiles)
    if has_streams:
        plan.set_streams(1)
    for cb, bb in itertools.product(chain_batches, band_blocks):
        plan.set_batch(cb)
        plan.set_band_block(bb)
        ms = _time_ms(lambda: plan.apply(psi, occ, want_ex=True), reps)
        table.append({"chain_batch": cb, "band_block": bb, "streams": 1, "tiles": list(tiles), "ms": ms})
    best = min(table, key=lambda r: r["ms"])
    plan.set_band_block(best["band_block"])
    best_streams = 1
    if has_streams:
        for ns, cb in itertools.product(streams, (best["chain_batch"], 2 * best["chain_batch"])):
            plan.set_streams(ns)
            plan.set_batch(cb)
            ms = _time_ms(lambda: plan.apply(psi, occ, want_ex=True), reps)
            row = {"chain_batch": cb, "band_block": best["band_block"], "streams": ns, "tiles": list(tiles), "ms": ms}
            table.append(row)
            if ms < best["ms"]:
                best, best_streams = row, ns
        plan.set_streams(best_streams)
    plan.set_batch(best["chain_batch"])
    best_ms = best["ms"]
    options = plan.tilings() if has_tiling else {}
    for p, name in enumerate(PASSES):
        if len(options.get(name, ())) < 2:
            continue
        trial = list(tiles)
        trial[p] = 1
        plan.set_tiling(trial)
        ms = _time_ms(lambda: plan.apply(psi, occ, want_ex=True), reps)
        table.append({"chain_batch": best["chain_batch"], "band_block": best["band_block"], "streams": best_streams,
                      "tiles": trial, "ms": ms})
        if ms < best_ms:
            tiles, best_ms = trial, ms
    if has_tiling:
        plan.set_tiling(tiles)
    res = {"chain_batch": best["chain_batch"], "band_block": best["band_block"], "streams": best_streams,
           "tiles": tiles, "ms": best_ms,
           "tiling": {name: dict(options[name][tiles[p]], tile=tiles[p])
                      for p, name in enumerate(PASSES) if name in options},
           "table": table}
    if use_cache:
        _store_cache(key, res)
    return res


def tune_batch(plans, psi, occ, slot_chains=(4, 8, 16), rings=(3, 4), ctas_per_sm=(0, 1),
               band_blocks=(16,), persistent=(1,), reps=1, use_cache=True, **fixed):
    """Fastest batch options for the systems ``plans``/``psi``/``occ``.

    Returns ``{"options": {...}, "ms": ..., "table": [...]}``; build the final
    batch with ``FockBatch(plans, psi, occ, **result["options"])``.
    """
    import torch
    shape = ",".join("%dx%d" % (p.grid[0], x.shape[0]) for p, x in zip(plans, psi))
    key = "batch|%s|prec%d|%s|%s" % (_gpu_name(), plans[0].precision, shape,
                                     json.dumps(fixed, sort_keys=True))
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            for p in plans:
                p.set_band_block(hit["band_block"])
                if hit.get("tiles") and hasattr(p, "tilings"):
                    t = p.tilings()
                    p.set_tiling([hit["tiles"][j] if len(t[name]) > 1 else 0 for j, name in enumerate(PASSES)])
            return dict(hit, cached=True)
    table = []
    combos = []
    for pers in persistent:
        if pers == 1:
            combos += [(bb, sc, ring, cps, 1) for bb, sc, ring, cps in
                       itertools.product(band_blocks, slot_chains, rings, ctas_per_sm)]
        elif pers == 2:  # dataflow launch: one CTA per task, no residency knob
            combos += [(bb, sc, ring, 0, 2) for bb, sc, ring in itertools.product(band_blocks, slot_chains, rings)]
        else:  # the persistent-launch knobs do not apply
            combos += [(bb, slot_chains[0], rings[0], 0, 0) for bb in band_blocks]
    for bb, sc, ring, cps, pers in combos:
        for p in plans:
            p.set_band_block(bb)
        opts = dict(fixed, slot_chains=sc, ring=ring, ctas_per_sm=cps, persistent=pers)
        b = FockBatch(plans, psi, occ, **opts)
        ms = _time_ms(b.run, reps)
        table.append({"band_block": bb, "options": opts, "ms": ms, "grid": b.info()["grid"]})
        b.close()
        torch.cuda.synchronize()
    best = min(table, key=lambda r: r["ms"])
    for p in plans:
        p.set_band_block(best["band_block"])
    # graph branches run each plan's own size-specialised kernels: try the
    # second FFT tiling of each pair pass on every plan that has one
    tiles = [0, 0, 0]
    best_ms = best["ms"]
    if not best["options"].get("persistent", 1) and all(hasattr(p, "tilings") for p in plans):
        two = [[len(p.tilings()[name]) > 1 for name in PASSES] for p in plans]
        for k in range(3):
            if not any(t[k] for t in two):
                continue
            trial = list(tiles)
            trial[k] = 1
            for p, t in zip(plans, two):
                p.set_tiling([trial[j] if t[j] else 0 for j in range(3)])
            b = FockBatch(plans, psi, occ, **best["options"])
            ms = _time_ms(b.run, reps)
            b.close()
            torch.cuda.synchronize()
            table.append({"band_block": best["band_block"], "options": best["options"], "tiles": trial, "ms": ms})
            if ms < best_ms:
                tiles, best_ms = trial, ms
        for p, t in zip(plans, two):
            p.set_tiling([tiles[j] if t[j] else 0 for j in range(3)])
    res = {"options": best["options"], "band_block": best["band_block"], "tiles": tiles, "ms": best_ms,
           "table": table}
    if use_cache:
        _store_cache(key, res)
    return res
