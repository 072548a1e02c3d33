"""The pair-block autotuner's search and cache (``autotune.py``) on the CPU:
candidate timings come from a fake clock, the plans and batches are stand-ins
that record what the tuner sets, so only the tuner's own logic runs."""

import json

import pytest

from paper_1305_7313_gb300 import autotune


class FakePlan:
    def __init__(self, n=96, precision=0):
        self.grid = (n, n, n)
        self.precision = precision
        self.chain_batch = None
        self.band_block = None
        self.applies = 0

    def set_batch(self, cb):
        self.chain_batch = cb

    def set_band_block(self, bb):
        self.band_block = bb

    def apply(self, psi, occ, want_ex=True):
        self.applies += 1


class FakeStreamPlan(FakePlan):
    """A plan that also takes a stream count."""

    def __init__(self, n=96, precision=0):
        super().__init__(n, precision)
        self.streams = None

    def set_streams(self, ns):
        self.streams = ns


class FakeTiledPlan(FakePlan):
    """A plan whose forward and inverse plane passes have two FFT tilings and
    whose column pass has one, as the library reports them."""

    def __init__(self):
        super().__init__()
        self.tiles = None

    def tilings(self):
        t0 = {"radices": [12, 8], "threads_per_line": 4, "threads": 384, "ntiles": 2}
        t1 = {"radices": [12, 4, 2], "threads_per_line": 8, "threads": 768, "ntiles": 2}
        one = {"radices": [12, 8], "threads_per_line": 4, "threads": 416, "ntiles": 1}
        return {"pair_fwd": [t0, t1], "pair_col": [one], "pair_inv": [t0, t1]}

    def set_tiling(self, tiles):
        self.tiles = list(tiles)


class FakePsi:
    def __init__(self, nb):
        self.shape = (nb, 100)


@pytest.fixture
def clock(monkeypatch, tmp_path):
    """Fake timer: the cost of a candidate is cost(state) for the state the
    tuner has set when it times; counts the timings."""
    monkeypatch.setenv("FOCK_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "fake GPU")
    state = {"calls": 0, "cost": None, "probe": None}

    def time_ms(fn, reps):
        state["calls"] += 1
        fn()
        return state["cost"](state["probe"]())

    monkeypatch.setattr(autotune, "_time_ms", time_ms)
    return state


def test_apply_tuner_times_every_candidate_and_keeps_the_fastest(clock):
    plan = FakePlan()
    cost = {(cb, bb): 100.0 + abs(cb - 19) + abs(bb - 16) for cb in (8, 17, 19, 32, 38) for bb in (8, 16, 32)}
    cost[(38, 8)] = 50.0  # the unique best
    clock["cost"] = lambda s: cost[s]
    clock["probe"] = lambda: (plan.chain_batch, plan.band_block)
    res = autotune.tune_apply(plan, FakePsi(512), None)
    assert (res["chain_batch"], res["band_block"], res["ms"]) == (38, 8, 50.0)
    assert (plan.chain_batch, plan.band_block) == (38, 8)  # left set on the plan
    assert len(res["table"]) == 15 and clock["calls"] == 15
    assert {(r["chain_batch"], r["band_block"]) for r in res["table"]} == set(cost)


def test_apply_tuner_cache_skips_the_search_and_is_keyed_by_workload(clock, tmp_path):
    clock["cost"] = lambda s: 10.0 if s == (17, 32) else 20.0
    p1 = FakePlan()
    clock["probe"] = lambda: (p1.chain_batch, p1.band_block)
    autotune.tune_apply(p1, FakePsi(64), None)
    n_search = clock["calls"]
    p2 = FakePlan()
    res = autotune.tune_apply(p2, FakePsi(64), None)
    assert res.get("cached") and clock["calls"] == n_search  # nothing timed again
    assert (p2.chain_batch, p2.band_block) == (17, 32)
    # another band count, grid size or precision is another key: searched anew
    for plan, nb in ((FakePlan(), 128), (FakePlan(n=48), 64), (FakePlan(precision=1), 64)):
        clock["probe"] = lambda plan=plan: (plan.chain_batch, plan.band_block)
        before = clock["calls"]
        assert not autotune.tune_apply(plan, FakePsi(nb), None).get("cached")
        assert clock["calls"] > before
    assert len(json.loads((tmp_path / "tune.json").read_text())) == 4


def test_a_corrupt_cache_file_is_ignored(clock, tmp_path):
    (tmp_path / "tune.json").write_text("{not json")
    plan = FakePlan()
    clock["cost"] = lambda s: float(s[0] * s[1])
    clock["probe"] = lambda: (plan.chain_batch, plan.band_block)
    res = autotune.tune_apply(plan, FakePsi(32), None, chain_batches=(4, 2), band_blocks=(3, 5))
    assert (res["chain_batch"], res["band_block"]) == (2, 3)
    assert json.loads((tmp_path / "tune.json").read_text())  # rewritten as valid JSON


def test_batch_tuner_candidates_and_choice(clock, monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    built = []

    class FakeBatch:
        def __init__(self, plans, psi, occ, **opts):
            self.opts = dict(opts, band_block=plans[0].band_block)
            built.append(self.opts)

        def run(self):
            pass

        def info(self):
            return {"grid": 152}

        def close(self):
            pass

    monkeypatch.setattr(autotune, "FockBatch", FakeBatch)
    clock["probe"] = lambda: built[-1]
    clock["cost"] = lambda o: 5.0 if (o["persistent"], o["slot_chains"], o["ring"], o["ctas_per_sm"]) == (1, 8, 4, 1) \
        else 9.0
    plans = [FakePlan(48), FakePlan(96)]
    res = autotune.tune_batch(plans, [FakePsi(10), FakePsi(20)], None, persistent=(1, 0, 2), band_blocks=(16,))
    # persistent candidates: every slot_chains x ring x ctas_per_sm; dataflow:
    # every slot_chains x ring; graph branches: one per band block
    assert len(built) == 3 * 2 * 2 + 1 + 3 * 2
    assert sum(1 for o in built if o["persistent"] == 0) == 1
    assert sum(1 for o in built if o["persistent"] == 2) == 6
    assert all(o["ctas_per_sm"] == 0 for o in built if o["persistent"] == 2)
    assert res["options"]["persistent"] == 1 and res["options"]["slot_chains"] == 8
    assert res["options"]["ring"] == 4 and res["options"]["ctas_per_sm"] == 1 and res["ms"] == 5.0
    assert all(p.band_block == 16 for p in plans)
    n = len(built)
    assert autotune.tune_batch(plans, [FakePsi(10), FakePsi(20)], None, persistent=(1, 0, 2),
                               band_blocks=(16,)).get("cached")
    assert len(built) == n


def test_apply_tuner_searches_the_fft_tilings_one_pass_at_a_time(clock):
    # pair-block grid at the default tiling, then each pass that has a second
    # tiling tried at the best block (the column pass has one: not tried);
    # the forward pass's second tiling is faster, the inverse pass's is not
    plan = FakeTiledPlan()
    def cost(s):
        cb, bb, tiles = s
        c = 100.0 + abs(cb - 19) + abs(bb - 16)
        if tiles[0] == 1:
            c -= 10.0
        if tiles[2] == 1:
            c += 5.0
        return c
    clock["cost"] = cost
    clock["probe"] = lambda: (plan.chain_batch, plan.band_block, tuple(plan.tiles))
    res = autotune.tune_apply(plan, FakePsi(512), None)
    assert (res["chain_batch"], res["band_block"], res["tiles"]) == (19, 16, [1, 0, 0])
    assert res["ms"] == 90.0 and plan.tiles == [1, 0, 0]
    assert clock["calls"] == 15 + 2  # 5 x 3 pair-block candidates, then two tilings
    assert res["tiling"]["pair_fwd"]["radices"] == [12, 4, 2] and res["tiling"]["pair_fwd"]["tile"] == 1
    assert res["tiling"]["pair_col"]["tile"] == 0 and res["tiling"]["pair_inv"]["tile"] == 0
    # a second process takes the choice from the cache without timing
    plan2 = FakeTiledPlan()
    res2 = autotune.tune_apply(plan2, FakePsi(512), None)
    assert res2["cached"] and plan2.tiles == [1, 0, 0] and clock["calls"] == 17


def test_apply_tuner_tries_stream_counts_with_the_best_and_twice_the_best_chain_batch(clock):
    plan = FakeStreamPlan()
    def cost(st):
        cb, bb, ns = st
        c = 100.0 + abs(cb - 19) + abs(bb - 16)
        if ns == 3 and cb == 38:
            c = 60.0  # three streams with twice the best single-stream batch
        elif ns > 1:
            c -= 5.0
        return c
    clock["cost"] = cost
    clock["probe"] = lambda: (plan.chain_batch, plan.band_block, plan.streams)
    res = autotune.tune_apply(plan, FakePsi(512), None)
    assert (res["chain_batch"], res["band_block"], res["streams"], res["ms"]) == (38, 16, 3, 60.0)
    assert (plan.chain_batch, plan.band_block, plan.streams) == (38, 16, 3)
    assert clock["calls"] == 15 + 3 * 2
    assert {(r["streams"], r["chain_batch"]) for r in res["table"] if r["streams"] > 1} == \
        {(ns, cb) for ns in (2, 3, 4) for cb in (19, 38)}
