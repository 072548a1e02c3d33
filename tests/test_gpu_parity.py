"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances:
* FP64 form and double-float form (FP64-class: ~48-bit significands, unit
  roundoff 2^-48 ~ 3.6e-15, so a transform chain of O(log Ntot) steps stays
  near 1e-13): 1e-10 relative (max |diff| / max |oracle|) on V_x psi and on
  E_x, the target of the FP64 path.
* mixed form (complex64 transforms): a transform of length Ntot in FP32 carries
  a relative error of a few u * log2(Ntot) with u = 2^-24 = 6e-8 and
  log2(Ntot) ~ 17-20, i.e. ~1e-6 RMS; the pair potential goes through two of
  them and a product, V_x psi through one more and an FP32 sum over bands.
  Bound used: 2e-5 on V_x psi (max norm), 5e-6 on E_x and dE_x/domega, whose
  terms are all non-negative and summed in FP64.
"""

import numpy as np
import pytest

import oracle
from oracle.kernels import ERFC as O_ERFC, SPENCER_ALAVI as O_SA
from paper_1305_7313_gb300 import FockPlan, synth
from paper_1305_7313_gb300 import _lib
from tests._common import cubic, rel_inf, require_gpu

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
FP64_FORMS = pytest.mark.parametrize("prec", [_lib.PREC_FP64, _lib.PREC_DF64], ids=["fp64", "df64"])
TOL32_V = 2e-5
TOL32_E = 5e-6


def setup_case(N, L, ecut, nb, seed, kind=_lib.SPENCER_ALAVI, omega=None, prec=_lib.PREC_FP64,
               occ=None, cell=None):
    torch = require_gpu()
    cell = cubic(L) if cell is None else np.asarray(cell, dtype=np.float64).ravel()
    plan = FockPlan(N, cell, ecut, kind, omega, prec)
    mill, _ = oracle.gsphere((N, N, N), cell, ecut)
    assert np.array_equal(plan.miller, mill)
    c = synth.orbitals(mill, cell, nb, seed)
    occ = np.full(nb, 2.0) if occ is None else np.asarray(occ, dtype=np.float64)
    psi = torch.from_numpy(c).cuda()
    return dict(torch=torch, plan=plan, mill=mill, c=c, occ=occ, psi=psi, cell=cell, N=N,
                kind=O_SA if kind == _lib.SPENCER_ALAVI else O_ERFC, omega=omega)


def oracle_of(case):
    return oracle.fock_apply(case["c"], case["occ"], case["mill"], (case["N"],) * 3, case["cell"],
                             case["kind"], case["omega"])


@FP64_FORMS
def test_small_fp64_matches_oracle(prec):
    # 24^3 grid, L = 10, Ecut = 10 Ha, 8 bands, f = 2, Spencer-Alavi
    case = setup_case(24, 10.0, 10.0, 8, 1305, prec=prec)
    vpsi, ex, _ = case["plan"].apply(case["psi"], case["occ"])
    vref, eref, _ = oracle_of(case)
    assert rel_inf(vpsi.cpu().numpy(), vref) <= TOL64
    assert abs(ex - eref) <= TOL64 * abs(eref)


@FP64_FORMS
def test_fp64_many_batches_ragged_tails_uneven_occupations(prec):
    # 48^3 grid, 37 bands (odd: a lone last pair and a lone last band), chains in
    # batches of 5 so both the pair loop and the band transforms have ragged tails
    occ = np.linspace(2.0, 0.0, 37)
    occ[5] = -0.5
    case = setup_case(48, 13.5, 12.0, 37, 77, occ=occ, prec=prec)
    case["plan"].set_batch(5)
    vpsi, ex, _ = case["plan"].apply(case["psi"], case["occ"])
    vref, eref, _ = oracle_of(case)
    assert rel_inf(vpsi.cpu().numpy(), vref) <= TOL64
    assert abs(ex - eref) <= TOL64 * abs(eref)


@FP64_FORMS
def test_fp64_erfc_energy_derivative_and_general_cell(prec):
    cell = np.array([[9.0, 0.4, 0.0], [0.3, 9.5, 0.2], [0.0, -0.3, 8.5]])
    case = setup_case(32, None, 8.0, 6, 5, kind=_lib.ERFC, omega=0.3, cell=cell,
                      occ=[2.0, 2.0, 1.5, 1.0, 0.5, 0.25], prec=prec)
    vpsi, ex, dex = case["plan"].apply(case["psi"], case["occ"], want_dex=True)
    vref, eref, dref = oracle_of(case)
    assert rel_inf(vpsi.cpu().numpy(), vref) <= TOL64
    assert abs(ex - eref) <= TOL64 * abs(eref)
    assert abs(dex - dref) <= TOL64 * abs(dref)


@FP64_FORMS
def test_single_band_and_two_bands(prec):
    for nb in (1, 2, 3):
        case = setup_case(24, 10.0, 10.0, nb, 40 + nb, prec=prec)
        vpsi, ex, _ = case["plan"].apply(case["psi"], case["occ"])
        vref, eref, _ = oracle_of(case)
        assert rel_inf(vpsi.cpu().numpy(), vref) <= TOL64
        assert abs(ex - eref) <= TOL64 * abs(eref)


@FP64_FORMS
def test_shards_sum_to_the_full_apply(prec):
    # the band-group split of the paper's EXX loop: partial results add up
    case = setup_case(24, 10.0, 10.0, 11, 9, prec=prec)
    vfull, efull, _ = case["plan"].apply(case["psi"], case["occ"])
    vsum = 0.0
    esum = 0.0
    for s in range(3):
        v, e, _ = case["plan"].apply_shard(case["psi"], case["occ"], s, 3)
        vsum = vsum + v.cpu().numpy()
        esum += e
    assert rel_inf(vsum, vfull.cpu().numpy()) <= 1e-13
    assert abs(esum - efull) <= 1e-13 * abs(efull)


@FP64_FORMS
def test_pair_energies_match_the_oracle(prec):
    case = setup_case(24, 10.0, 10.0, 6, 21, kind=_lib.ERFC, omega=0.4, prec=prec)
    pairs = [(0, 0), (0, 5), (3, 2), (4, 4), (1, 3)]
    e, d = case["plan"].pair_energies(case["psi"], pairs, want_d=True)
    psi = oracle.orbitals_to_real(case["c"], case["mill"], (24,) * 3, case["cell"], real=True)
    from oracle.fock import kernel_grid
    vg, dvg = kernel_grid(O_ERFC, (24,) * 3, case["cell"], 0.4)
    for k, (i, j) in enumerate(pairs):
        er, dr = oracle.pair_energy(psi[i], psi[j], vg, dvg)
        assert abs(e[k] - er) <= TOL64 * abs(er)
        assert abs(d[k] - dr) <= TOL64 * abs(dr)


def test_mixed_precision_matches_oracle_within_stated_bound():
    case = setup_case(48, 13.5, 12.0, 20, 31, kind=_lib.ERFC, omega=0.106, prec=_lib.PREC_MIXED32)
    vpsi, ex, dex = case["plan"].apply(case["psi"], case["occ"], want_dex=True)
    vref, eref, dref = oracle_of(case)
    assert rel_inf(vpsi.cpu().numpy(), vref) <= TOL32_V
    assert abs(ex - eref) <= TOL32_E * abs(eref)
    assert abs(dex - dref) <= TOL32_E * abs(dref)


def test_invalid_calls_fail_cleanly():
    case = setup_case(24, 10.0, 10.0, 4, 3)
    torch = case["torch"]
    plan = case["plan"]
    with pytest.raises(_lib.FockError) as e:
        _lib.fock_apply(plan.handle, case["psi"], case["occ"], case["psi"])  # in place
    assert e.value.status == 1
    with pytest.raises(_lib.FockError):
        _lib.fock_apply_shard(plan.handle, case["psi"], case["occ"], 3, 3, torch.empty_like(case["psi"]))
    with pytest.raises(_lib.FockError):
        _lib.fock_apply(plan.handle, case["psi"], [2.0, np.nan, 2.0, 2.0], torch.empty_like(case["psi"]))
    with pytest.raises(_lib.FockError):
        plan.pair_energies(case["psi"], [(0, 4)])
    # the plan still works afterwards
    vpsi, ex, _ = plan.apply(case["psi"], case["occ"])
    vref, eref, _ = oracle_of(case)
    assert abs(ex - eref) <= TOL64 * abs(eref)


@pytest.mark.parametrize("prec", [_lib.PREC_FP64, _lib.PREC_DF64, _lib.PREC_MIXED32],
                         ids=["fp64", "df64", "mixed32"])
def test_empty_occupations_give_zero_and_no_bands_is_refused(prec):
    # every f_i = 0: each term of V_x psi and of E_x carries an occupation, so
    # both are exactly zero (the uniform-occupation scaling and the mixed
    # form's FP64 overlaps included); a call with no bands is an error
    torch = require_gpu()
    case = setup_case(24, 10.0, 10.0, 7, 17, kind=_lib.ERFC, omega=0.3, prec=prec, occ=np.zeros(7))
    plan = case["plan"]
    vpsi = torch.full_like(case["psi"], complex(np.nan, np.nan))
    ex, dex = _lib.fock_apply(plan.handle, case["psi"], case["occ"], vpsi, want_dex=True)
    assert ex == 0.0 and dex == 0.0
    assert bool(torch.all(vpsi == 0).item())  # written (no NaN left) and zero
    vref, eref, dref = oracle_of(case)
    assert not np.any(vref) and eref == 0.0 and dref == 0.0
    with pytest.raises(_lib.FockError):
        _lib.fock_apply(plan.handle, case["psi"][:0], [], torch.empty_like(case["psi"][:0]))
    # the plan still works afterwards, with occupations again
    case["occ"] = np.full(7, 2.0)
    v2, e2, _ = plan.apply(case["psi"], case["occ"])
    vref, eref, _ = oracle_of(case)
    tol_v, tol_e = (TOL32_V, TOL32_E) if prec == _lib.PREC_MIXED32 else (TOL64, TOL64)
    assert rel_inf(v2.cpu().numpy(), vref) <= tol_v
    assert abs(e2 - eref) <= tol_e * abs(eref)


@pytest.mark.parametrize("prec,tol_v,tol_e", [(_lib.PREC_FP64, TOL64, TOL64), (_lib.PREC_DF64, TOL64, TOL64),
                                              (_lib.PREC_MIXED32, TOL32_V, TOL32_E)],
                         ids=["fp64", "df64", "mixed32"])
@pytest.mark.parametrize("N", [8, 12, 16, 36, 64, 72])
def test_every_other_compiled_size_in_every_form(N, prec, tol_v, tol_e):
    # the grid sizes the tests above do not reach (24, 32, 48 are covered),
    # each with its own radix plan (8 and 12 in one stage, 16 = 4 x 4 in
    # registers, 36 = 6 x 6, 64 = 8 x 8, 72 = 12 x 6): cells with L = 0.3 N
    # bohr and Ecut = 6 Ha, a few unevenly occupied bands
    nb = 5 if N <= 36 else 3
    case = setup_case(N, 0.3 * N, 6.0, nb, 500 + N, prec=prec, occ=np.linspace(2.0, 1.0, nb))
    vpsi, ex, _ = case["plan"].apply(case["psi"], case["occ"])
    vref, eref, _ = oracle_of(case)
    assert rel_inf(vpsi.cpu().numpy(), vref) <= tol_v
    assert abs(ex - eref) <= tol_e * abs(eref)


def test_double_float_form_refused_where_not_built():
    torch = require_gpu()
    with pytest.raises(_lib.FockError):
        _lib.fock_kplan_create((16, 16, 16), cubic(7.0), 6.0, [[0.0, 0.0, 0.0]], [1.0], _lib.ERFC, (0.5,),
                               _lib.PREC_DF64)


def test_orbitals_of_another_sphere_are_refused_before_any_device_work():
    case = setup_case(24, 10.0, 10.0, 3, 7)
    torch = case["torch"]
    wrong = torch.zeros((3, case["psi"].shape[1] - 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError, match="plan's sphere"):
        case["plan"].apply(wrong, case["occ"])
    vpsi, ex, _ = case["plan"].apply(case["psi"], case["occ"])  # the plan still works
    assert np.isfinite(ex)


@pytest.mark.parametrize("prec,kind,omega,tol_v,tol_e", [
    (_lib.PREC_FP64, _lib.SPENCER_ALAVI, None, TOL64, TOL64),
    (_lib.PREC_MIXED32, _lib.ERFC, 0.106, TOL32_V, TOL32_E),
], ids=["fp64", "mixed32"])
def test_every_fft_tiling_matches_the_oracle(prec, kind, omega, tol_v, tol_e):
    # 96^3 at L = 27, Ecut = 12 (the grid with two compiled tilings), 6 bands:
    # every combination of the passes' tilings against the oracle, and the
    # tuner's choice list as the library describes it
    import itertools
    case = setup_case(96, 27.0, 12.0, 6, 4096, kind=kind, omega=omega, prec=prec)
    plan = case["plan"]
    tilings = plan.tilings()
    assert [len(tilings[p]) for p in _lib.PASSES] == [2, 2, 2]
    for p in _lib.PASSES:
        t0, t1 = tilings[p]
        assert t0["radices"] != t1["radices"] and t0["threads_per_line"] != t1["threads_per_line"]
        assert int(np.prod(t0["radices"])) == int(np.prod(t1["radices"])) == 96
    vref, eref, _ = oracle_of(case)
    for tiles in itertools.product((0, 1), repeat=3):
        plan.set_tiling(tiles)
        vpsi, ex, _ = plan.apply(case["psi"], case["occ"])
        assert rel_inf(vpsi.cpu().numpy(), vref) <= tol_v, tiles
        assert abs(ex - eref) <= tol_e * abs(eref), tiles
    with pytest.raises(_lib.FockError):
        plan.set_tiling((2, 0, 0))
    plan.close()


def test_a_grid_with_one_tiling_refuses_the_second():
    case = setup_case(24, 10.0, 10.0, 4, 17, prec=_lib.PREC_MIXED32, kind=_lib.ERFC, omega=0.5)
    plan = case["plan"]
    assert all(len(v) == 1 for v in plan.tilings().values())
    with pytest.raises(_lib.FockError):
        plan.set_tiling((1, 0, 0))
    plan.set_tiling((0, 0, 0))
    plan.close()


@pytest.mark.parametrize("prec,tol", [(_lib.PREC_FP64, TOL64), (_lib.PREC_MIXED32, TOL32_V),
                                      (_lib.PREC_DF64, TOL64)], ids=["fp64", "mixed32", "df64"])
def test_pair_launches_on_several_streams_match_the_oracle(prec, tol):
    # small launches (5 chains of 36 pairs' 18 chains) rotated over 1-4 streams,
    # each with its own transform buffer; deterministic accumulation too (FP64
    # forms): the same bits on every stream count
    case = setup_case(24, 10.0, 10.0, 8, 1305, prec=prec)
    plan = case["plan"]
    plan.set_batch(5)
    vref, eref, _ = oracle_of(case)
    for streams in (1, 2, 3, 4):
        plan.set_streams(streams)
        vpsi, ex, _ = plan.apply(case["psi"], case["occ"])
        assert rel_inf(vpsi.cpu().numpy(), vref) <= tol, streams
        assert abs(ex - eref) <= (TOL64 if prec != _lib.PREC_MIXED32 else TOL32_E) * abs(eref), streams
    if prec != _lib.PREC_MIXED32:
        plan.set_deterministic(True)
        bits = []
        for streams in (1, 3):
            plan.set_streams(streams)
            vpsi, ex, _ = plan.apply(case["psi"], case["occ"])
            bits.append((vpsi.cpu().numpy().tobytes(), ex))
        assert bits[0] == bits[1]
    with pytest.raises(_lib.FockError):
        plan.set_streams(5)
    plan.close()


@pytest.mark.parametrize("kind,omega", [(_lib.SPENCER_ALAVI, None), (_lib.ERFC, 0.3)], ids=["sa", "erfc"])
def test_mixed_form_takes_the_g0_term_from_fp64_overlaps(kind, omega):
    # one band c(G) = delta_G0, psi(r) = Omega^-1/2: the pair density is a
    # constant, its transform vanishes away from G = 0 in any arithmetic, and
    # the one kernel term, at G = 0, comes from the FP64 overlap of the pair's
    # coefficients: E_x and dE_x/domega to FP64 rounding (the FP32 transform's
    # own G = 0 value is good to ~1e-7 only)
    torch = require_gpu()
    N, L, ecut = 32, 11.0, 6.0
    cell = cubic(L)
    plan = FockPlan(N, cell, ecut, kind, omega, _lib.PREC_MIXED32)
    mill, _ = oracle.gsphere((N,) * 3, cell, ecut)
    c = np.zeros((1, len(mill)), dtype=np.complex128)
    c[0, int(np.flatnonzero(np.all(mill == 0, axis=1))[0])] = 1.0
    occ = np.array([2.0])
    want_d = kind == _lib.ERFC
    vpsi, ex, dex = plan.apply(torch.from_numpy(c).cuda(), occ, want_dex=want_d)
    ok = O_SA if kind == _lib.SPENCER_ALAVI else O_ERFC
    _, eref, dref = oracle.fock_apply(c, occ, mill, (N,) * 3, cell, ok, omega)
    assert abs(ex - eref) <= 1e-13 * abs(eref)
    if want_d:
        assert abs(dex - dref) <= 1e-13 * abs(dref)
    plan.close()
