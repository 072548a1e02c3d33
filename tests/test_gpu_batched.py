"""Batched form: uneven systems in one persistent pair launch under a CUDA
graph, against single-system applies (themselves parity-tested) and the FP64
oracle; and the bounded-wait failure path."""

import numpy as np
import pytest

import oracle
from paper_1305_7313_gb300 import FockBatch, FockPlan, _lib, synth
from tests._common import cubic, rel_inf, require_gpu

pytestmark = pytest.mark.gpu

# (N, L, Ecut, nb): uneven grids and band counts, two systems share a grid size
SYSTEMS = [(24, 10.0, 10.0, 5), (32, 9.0, 12.0, 9), (48, 13.5, 12.0, 12), (24, 8.0, 8.0, 3)]


def make_systems(prec, kind=_lib.SPENCER_ALAVI, omega=None, seed=50):
    torch = require_gpu()
    plans, psis, occs, cs = [], [], [], []
    for k, (n, L, ecut, nb) in enumerate(SYSTEMS):
        p = FockPlan(n, cubic(L), ecut, kind, omega, prec)
        c = synth.orbitals(p.miller, cubic(L), nb, seed + k)
        plans.append(p)
        cs.append(c)
        psis.append(torch.from_numpy(c).cuda())
        occs.append(np.linspace(2.0, 1.0, nb))
    return torch, plans, psis, occs, cs


@pytest.mark.parametrize("prec,tol_v,tol_e", [(_lib.PREC_FP64, 1e-10, 1e-10),
                                              (_lib.PREC_MIXED32, 2e-5, 5e-6)])
@pytest.mark.parametrize("use_graph,persistent", [(1, 1), (0, 1), (1, 0), (1, 2), (0, 2)])
def test_batch_matches_single_applies_and_oracle(prec, tol_v, tol_e, use_graph, persistent):
    torch, plans, psis, occs, cs = make_systems(prec, _lib.ERFC, 0.3)
    singles = []
    for p, psi, occ in zip(plans, psis, occs):
        v, e, d = p.apply(psi, occ, want_dex=True)
        singles.append((v.cpu().numpy(), e, d))
    # small slots force many segments, slot reuse across systems and ragged runs
    for p in plans:
        p.set_batch(3)  # several launches per system in the non-persistent mode
    batch = FockBatch(plans, psis, occs, slot_chains=2, ring=3, use_graph=use_graph, want_dex=1,
                      persistent=persistent)
    info = batch.info()
    assert info["segments"] > 3 * len(SYSTEMS)
    for _ in range(2):  # replay
        ex, dex = batch.run()
        assert batch.info()["persist_ms"] > 0.0
        for k in range(len(SYSTEMS)):
            v = batch.vpsi[k].cpu().numpy()
            assert rel_inf(v, singles[k][0]) <= tol_v
            assert abs(ex[k] - singles[k][1]) <= tol_e * abs(singles[k][1])
            assert abs(dex[k] - singles[k][2]) <= tol_e * abs(singles[k][2])
    for k in (0, 3):
        n, L, ecut, nb = SYSTEMS[k]
        vref, eref, dref = oracle.fock_apply(cs[k], occs[k], plans[k].miller, (n, n, n), cubic(L), "erfc", 0.3)
        assert rel_inf(batch.vpsi[k].cpu().numpy(), vref) <= tol_v
        assert abs(ex[k] - eref) <= tol_e * abs(eref)
    batch.close()


def test_batch_input_update_between_replays():
    torch, plans, psis, occs, cs = make_systems(_lib.PREC_FP64)
    batch = FockBatch(plans, psis, occs)
    ex1, _ = batch.run()
    # new orbitals written in place into the captured buffer of system 1
    c_new = synth.orbitals(plans[1].miller, cubic(SYSTEMS[1][1]), SYSTEMS[1][3], 999)
    psis[1].copy_(torch.from_numpy(c_new))
    ex2, _ = batch.run()
    assert ex2[0] == pytest.approx(ex1[0], rel=1e-12)
    n, L, ecut, nb = SYSTEMS[1]
    _, eref, _ = oracle.fock_apply(c_new, occs[1], plans[1].miller, (n, n, n), cubic(L), "spencer_alavi")
    assert abs(ex2[1] - eref) <= 1e-10 * abs(eref)
    batch.close()


@pytest.mark.parametrize("persistent", [1, 2])
def test_a_wait_that_never_ends_times_out_and_the_device_stays_usable(persistent):
    torch, plans, psis, occs, cs = make_systems(_lib.PREC_MIXED32)
    # segment 4 waits for its own completion: nothing will ever set that counter
    stalled = FockBatch(plans, psis, occs, slot_chains=2, wait_limit_s=0.5, stall_segment=4, persistent=persistent)
    with pytest.raises(_lib.FockError) as err:
        stalled.run()
    assert err.value.status == 6  # FOCK_ERR_TIMEOUT
    stalled.close()
    torch.cuda.synchronize()
    ok = FockBatch(plans, psis, occs, slot_chains=2, persistent=persistent)
    ex, _ = ok.run()
    e0 = plans[0].apply(psis[0], occs[0])[1]
    assert abs(ex[0] - e0) <= 5e-6 * abs(e0)
    ok.close()


def test_batch_rejects_bad_input():
    torch, plans, psis, occs, cs = make_systems(_lib.PREC_FP64)
    with pytest.raises(_lib.FockError):
        FockBatch([plans[0], plans[0]], [psis[0], psis[0]], [occs[0], occs[0]])  # same plan twice
    with pytest.raises(_lib.FockError):
        FockBatch(plans[:2], psis[:2], occs[:2], ring=2)
    p16 = FockPlan(16, cubic(8.0), 4.0)
    c16 = torch.from_numpy(synth.orbitals(p16.miller, cubic(8.0), 2, 1)).cuda()
    with pytest.raises(_lib.FockError) as err:
        FockBatch([p16], [c16], [np.ones(2)])
    assert err.value.status == 2


def test_autotuner_picks_a_candidate_and_keeps_results(tmp_path, monkeypatch):
    monkeypatch.setenv("FOCK_TUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_1305_7313_gb300.autotune import tune_apply, tune_batch
    torch, plans, psis, occs, cs = make_systems(_lib.PREC_MIXED32)
    v0, e0, _ = plans[2].apply(psis[2], occs[2])
    v0 = v0.cpu().numpy()
    r = tune_apply(plans[2], psis[2], occs[2], chain_batches=(2, 5), band_blocks=(4, 16), reps=1)
    # the pair-block grid on one stream, then 2-4 streams with the best chain
    # batch and twice it (48^3 has one FFT tiling per pass: none searched)
    best1 = min((row for row in r["table"] if row["streams"] == 1), key=lambda row: row["ms"])
    assert (r["chain_batch"], r["band_block"]) in [(cb, best1["band_block"]) for cb in
                                                   (best1["chain_batch"], 2 * best1["chain_batch"])] + \
        [(best1["chain_batch"], best1["band_block"])]
    assert len(r["table"]) == 4 + 3 * 2 and r["streams"] in (1, 2, 3, 4)
    v1, e1, _ = plans[2].apply(psis[2], occs[2])
    assert rel_inf(v1.cpu().numpy(), v0) <= 2e-5 and abs(e1 - e0) <= 5e-6 * abs(e0)
    again = tune_apply(plans[2], psis[2], occs[2], chain_batches=(2, 5), band_blocks=(4, 16))
    assert again.get("cached") and again["chain_batch"] == r["chain_batch"]
    rb = tune_batch(plans, psis, occs, slot_chains=(1, 3), rings=(3, 4), ctas_per_sm=(0,))
    assert len(rb["table"]) == 4
    b = FockBatch(plans, psis, occs, **rb["options"])
    ex, _ = b.run()
    assert abs(ex[2] - e0) <= 5e-6 * abs(e0)
    b.close()


@pytest.mark.parametrize("persistent", [0, 2])
def test_the_full_sixteen_system_batch_matches_single_applies(persistent):
    # the benchmark's batch: 16 systems on 48^3, 64^3, 72^3 and 96^3 grids
    # (L = 27 N / 96, Ecut 12 Ha, 32-384 bands, 298,602 pairs), mixed form:
    # E_x of every system and V_x psi of the last band of one system per grid
    # size against the same systems applied one at a time
    from paper_1305_7313_gb300.workloads import batched_systems, cubic_cell
    torch = require_gpu()
    systems = batched_systems()
    plans, psis, occs = [], [], []
    for sy in systems:
        p = FockPlan(sy["N"], cubic_cell(sy["L"]), sy["ecut"], sy["kernel"], sy["omega"], sy["prec"])
        c = synth.orbitals(p.miller, cubic_cell(sy["L"]), sy["nb"], sy["seed"])
        plans.append(p)
        psis.append(torch.from_numpy(c).cuda())
        occs.append(np.full(sy["nb"], 2.0))
    assert sum(sy["nb"] * (sy["nb"] + 1) // 2 for sy in systems) == 298602
    batch = FockBatch(plans, psis, occs, persistent=persistent, slot_chains=16)
    ex, _ = batch.run()
    first_of_size = {}
    for k, sy in enumerate(systems):
        first_of_size.setdefault(sy["N"], k)
    for k, sy in enumerate(systems):
        v, e, _ = plans[k].apply(psis[k], occs[k])
        assert abs(ex[k] - e) <= 5e-6 * abs(e), (k, sy["N"])
        if first_of_size[sy["N"]] == k:
            last = sy["nb"] - 1
            assert rel_inf(batch.vpsi[k][last].cpu().numpy(), v[last].cpu().numpy()) <= 2e-5, (k, sy["N"])
        del v
    batch.close()
    for p in plans:
        p.close()
    torch.cuda.empty_cache()
