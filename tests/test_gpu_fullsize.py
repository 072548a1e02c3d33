"""The 96^3 / 512-band workloads (L = 27 bohr, Ecut = 12 Ha, 39,127 plane
waves, all 131,328 unique pairs) in the launch configurations the benchmark
times, against outputs the oracle computes one by one — V_x psi of the last
band (the ragged end of the pair schedule) and a sample of pair energies — and
against properties that hold at any size: <psi_a|V_x|psi_b> Hermitian and
negative semidefinite, and E_x = 1/2 sum_j f_j <psi_j|V_x psi_j> between the
energy the column pass sums and the one V_x psi implies.

The oracle's share costs about a minute of host time per kernel (one band
against all 512, plus the real-space orbitals)."""

import numpy as np
import pytest

import oracle
from oracle.fock import kernel_grid
from paper_1305_7313_gb300 import FockPlan, _lib, synth
from paper_1305_7313_gb300.workloads import WORKLOADS, cubic_cell
from tests._common import require_gpu

pytestmark = pytest.mark.gpu

N = 96
GRID = (N, N, N)
LAST = 511
PAIRS = [(0, 0), (0, 511), (17, 300), (255, 256), (511, 511), (100, 400), (3, 4)]

# (workload, precision, [(chain_batch, band_block)], tolerance on V_x psi, on E_x)
FORMS = {
    "fp64": ("gamma_fp64_L27_N96_nb512", _lib.PREC_FP64, [(None, None), (17, 8)], 1e-10, 1e-10),
    "df64": ("gamma_df64_L27_N96_nb512", _lib.PREC_DF64, [(None, None)], 1e-10, 1e-10),
    "mixed32": ("gamma_mixed32_erfc_L27_N96_nb512", _lib.PREC_MIXED32, [(None, None), (32, 8)], 2e-5, 5e-6),
}

_REF = {}


def reference(name):
    """Oracle V_x psi of band LAST and the energies of PAIRS for workload `name`."""
    w = WORKLOADS[name]
    key = (w["seed"], w["kernel"], w["omega"])
    if key in _REF:
        return _REF[key]
    cell = np.asarray(cubic_cell(w["L"]))
    mill, _ = oracle.gsphere(GRID, cell, w["ecut"])
    c = synth.orbitals(mill, cell, w["nb"], w["seed"])
    occ = np.full(w["nb"], 2.0)
    kind = "spencer_alavi" if w["kernel"] == _lib.SPENCER_ALAVI else "erfc"
    psi = oracle.orbitals_to_real(c, mill, GRID, cell, real=True)
    vlast, _, _ = oracle.fock_apply(c, occ, mill, GRID, cell, kind, w["omega"], out_bands=[LAST], psi=psi)
    vg, dvg = kernel_grid(kind, GRID, cell, w["omega"])
    epairs = [oracle.pair_energy(psi[i], psi[j], vg) for i, j in PAIRS]
    del psi
    _REF[key] = dict(c=c, occ=occ, mill=mill, cell=cell, kind=w["kernel"], omega=w["omega"], vlast=vlast[0],
                      epairs=np.array(epairs), ecut=w["ecut"])
    return _REF[key]


@pytest.mark.parametrize("form", list(FORMS))
def test_full_size_against_sampled_oracle_outputs_and_invariants(form):
    torch = require_gpu()
    name, prec, configs, tol_v, tol_e = FORMS[form]
    ref = reference(name)
    plan = FockPlan(N, ref["cell"], ref["ecut"], ref["kind"], ref["omega"], prec)
    assert np.array_equal(plan.miller, ref["mill"])
    psi = torch.from_numpy(ref["c"]).cuda()
    occ = ref["occ"]
    vmax = np.max(np.abs(ref["vlast"]))
    for cb, bb in configs:
        if cb is not None:
            plan.set_batch(cb)
            plan.set_band_block(bb)
        vpsi, ex, _ = plan.apply(psi, occ)
        # sampled output: V_x psi of the last band, element by element
        assert np.max(np.abs(vpsi[LAST].cpu().numpy() - ref["vlast"])) <= tol_v * vmax
        # invariants over all 512 bands, on the device in FP64
        m = psi.conj() @ vpsi.T  # M_ab = <psi_a | V_x psi_b>
        mnorm = float(m.abs().max())
        assert float((m - m.conj().T).abs().max()) <= (1e-12 if tol_v <= 1e-10 else 1e-5) * mnorm
        ev = torch.linalg.eigvalsh(0.5 * (m + m.conj().T))
        assert float(ev.max()) <= (1e-10 if tol_v <= 1e-10 else 1e-5) * mnorm
        e_from_v = 0.5 * float((torch.from_numpy(occ).cuda() * torch.diagonal(m).real).sum())
        assert abs(ex - e_from_v) <= tol_e * abs(ex)
    # sampled pair energies, one by one
    e = plan.pair_energies(psi, PAIRS)
    assert np.max(np.abs(np.asarray(e) - ref["epairs"]) / np.abs(ref["epairs"])) <= tol_e
    plan.close()
    del psi, vpsi, m
    torch.cuda.empty_cache()


@pytest.mark.parametrize("form", list(FORMS))
def test_first_64_bands_match_the_stored_oracle_energy(form):
    # E_x (and dE_x/domega for the erfc kernel) of the first 64 bands of the
    # 96^3 workloads against the oracle's values over the same 64 bands
    # (tests/golden/oracle_fullsize_N96_nb64.txt, written from oracle/ alone),
    # plus V_x psi of three bands at 203 sampled sphere positions each
    from tests.golden import fullsize_record
    torch = require_gpu()
    name, prec, _, tol_v, tol_e = FORMS[form]
    w = WORKLOADS[name]
    rec = fullsize_record.load()
    case = fullsize_record.CASE_OF_SEED[w["seed"]]
    cell = np.asarray(cubic_cell(w["L"]))
    plan = FockPlan(N, cell, w["ecut"], w["kernel"], w["omega"], prec)
    assert plan.npw == rec["npw"]
    c = synth.orbitals(plan.miller, cell, w["nb"], w["seed"])[:fullsize_record.NB]
    psi = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    vpsi, ex, dex = plan.apply(psi, np.full(fullsize_record.NB, 2.0), want_dex=True)
    err = fullsize_record.compare(rec, case, ex, dex, vpsi.cpu().numpy())
    assert err["rel_dEx"] <= tol_e, err
    if err["rel_ddEx_domega"] is not None:
        assert err["rel_ddEx_domega"] <= tol_e, err
    assert err["max_abs_dVpsi_rel"] <= tol_v, err
    plan.close()
