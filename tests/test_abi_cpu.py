"""The C-ABI library on a machine without a GPU: it loads, exports every
declared entry point, and its host-only logic (status strings, argument checks,
the plane-wave sphere) behaves as documented.  No compute call is made."""

import ctypes

import numpy as np
import pytest

import oracle
from paper_1305_7313_gb300 import _lib
from tests._common import built_library, cubic, declared_functions


@pytest.fixture(scope="module")
def lib():
    return built_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib._SIGNATURES)


def test_status_strings(lib):
    for code in range(7):
        s = _lib.fock_status_string(code)
        assert s and s != "unknown status"
    assert _lib.fock_status_string(99) == "unknown status"


@pytest.mark.parametrize("grid,L,ecut,npw", [
    ((24, 24, 24), 10.0, 10.0, 1503),
    ((96, 96, 96), 27.0, 12.0, 39127),
    ((72, 72, 72), 20.0, 12.0, 15895),
    ((48, 48, 48), 13.5, 12.0, None),
])
def test_sphere_is_bit_identical_to_the_oracle(lib, grid, L, ecut, npw):
    m = _lib.fock_gsphere(grid, cubic(L), ecut)
    mo, _ = oracle.gsphere(grid, cubic(L), ecut)
    if npw is not None:
        assert len(m) == npw
    assert m.dtype == np.int32 and np.array_equal(m, mo)


def test_sphere_general_cell_bit_identical(lib):
    cells = [
        np.array([[7.0, 0.3, 0.0], [0.5, 8.0, 0.2], [0.0, -0.4, 6.5]]),
        np.array([[6.0, 0.0, 0.0], [3.0, 5.196152422706632, 0.0], [0.0, 0.0, 9.0]]),  # hexagonal
        np.array([[0.0, 5.0, 5.0], [5.0, 0.0, 5.0], [5.0, 5.0, 0.0]]),                # fcc
    ]
    for c in cells:
        m = _lib.fock_gsphere((32, 32, 32), c.ravel(), 7.0)
        mo, _ = oracle.gsphere((32, 32, 32), c.ravel(), 7.0)
        assert np.array_equal(m, mo)


def test_sphere_errors(lib):
    with pytest.raises(_lib.FockError) as e:
        _lib.fock_gsphere((12, 12, 12), cubic(10.0), 10.0)
    assert e.value.status == 3
    with pytest.raises(_lib.FockError) as e:
        _lib.fock_gsphere((24, 24, 24), cubic(10.0), -1.0)
    assert e.value.status == 1
    with pytest.raises(_lib.FockError) as e:
        _lib.fock_gsphere((24, 24, 24), np.zeros(9), 1.0)
    assert e.value.status == 1
    n = ctypes.c_int64()
    g = (ctypes.c_int * 3)(24, 24, 24)
    cell = np.ascontiguousarray(cubic(10.0))
    buf = np.empty((10, 3), dtype=np.int32)
    st = lib.fock_gsphere(g, cell.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 10.0,
                          ctypes.byref(n), buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 10)
    assert st == 1 and n.value == 1503


@pytest.mark.parametrize("grid,kind,kp,prec,flags,status", [
    ((24, 24, 20), 0, (), 0, 1, 2),      # not cubic
    ((20, 20, 20), 0, (), 0, 1, 2),      # N = 20 has a factor 5
    ((120, 120, 120), 0, (), 0, 1, 2),   # no kernels compiled for this N
    ((24, 24, 24), 1, (), 0, 1, 1),      # erfc without omega
    ((24, 24, 24), 1, (-1.0,), 0, 1, 1),  # negative omega
    ((24, 24, 24), 0, (), 0, 0, 1),      # FOCK_GAMMA_REAL missing
    ((24, 24, 24), 0, (), 7, 1, 1),      # unknown precision
    ((24, 24, 24), 5, (), 0, 1, 1),      # unknown kernel
    ((12, 12, 12), 0, (), 0, 1, 3),      # sphere does not fit
])
def test_plan_create_rejects_bad_arguments_before_touching_the_gpu(lib, grid, kind, kp, prec, flags, status):
    with pytest.raises(_lib.FockError) as e:
        _lib.fock_plan_create(grid, cubic(10.0), 10.0, kind, kp, prec, flags)
    assert e.value.status == status
    assert _lib.fock_last_error(None) != ""


def test_null_arguments_are_rejected(lib):
    assert lib.fock_plan_create(None, None, None, 1.0, 0, None, 0, 0, 1) == 1
    assert lib.fock_plan_npw(None, None) == 1
    assert lib.fock_apply(None, None, 1, None, None, None, None, None) == 1
    assert lib.fock_destroy(None) == 0
    assert lib.fock_plan_set_batch(None, 4) == 1


STRING_ENTRIES = {"fock_status_string", "fock_last_error", "fock_batch_last_error", "fock_kplan_last_error"}


def _zero_args(argtypes):
    return [0.0 if t is ctypes.c_double else (0 if t in (ctypes.c_int, ctypes.c_uint, ctypes.c_int64) else None)
            for t in argtypes]


def test_every_entry_point_rejects_null_handles_and_pointers(lib):
    # the header's shared rule: a NULL handle or pointer (or a zero where a
    # count must be positive) is INVALID_ARG, the *_destroy calls accept NULL;
    # nothing reaches the GPU, so this runs without one
    for name, argtypes in _lib._SIGNATURES.items():
        if name in STRING_ENTRIES:
            continue
        st = getattr(lib, name)(*_zero_args(argtypes))
        expect = 0 if name.endswith("_destroy") else 1
        assert st == expect, (name, _lib.STATUS.get(st, st))


def test_error_text_entries_accept_null_handles(lib):
    for name in ("fock_last_error", "fock_batch_last_error", "fock_kplan_last_error"):
        assert isinstance(getattr(lib, name)(None), bytes)


def test_kpoint_spheres_are_bit_identical_to_the_oracle(lib):
    cells = [np.diag([7.0, 7.0, 7.0]), np.array([[6.0, 0.4, 0.0], [0.0, 6.5, 0.3], [0.2, 0.0, 5.5]])]
    for cell in cells:
        for kf in [(0.0, 0.0, 0.0), (0.5, 0.0, 0.0), (0.25, -0.25, 0.5), (1.0 / 3.0, 0.1, -0.45)]:
            m = _lib.fock_gsphere_k((24, 24, 24), cell.ravel(), 6.0, kf)
            mo, _ = oracle.gsphere_k((24, 24, 24), cell.ravel(), 6.0, kf)
            assert np.array_equal(m, mo)


def _pair_density_reach(grid, cell, ecut, kpts):
    # largest frequency difference m_b - m_a between two spheres of the mesh
    lo, hi = [], []
    for k in kpts:
        m, _ = oracle.gsphere_k(grid, cell, ecut, k)
        lo.append(m.min(0))
        hi.append(m.max(0))
    return max(int((hi[b] - lo[a]).max()) for a in range(len(kpts)) for b in range(len(kpts)))


@pytest.mark.parametrize("n,L,ecut,kpts,refused", [
    (16, 7.0, 6.0, [[0, 0, 0], [0.5, 0, 0], [0, 0.5, 0.5], [0.25, -0.25, 0.5]], True),
    (16, 7.0, 4.0, [[0, 0, 0], [0.5, 0, 0], [0, 0.5, 0.5], [0.25, -0.25, 0.5]], False),
    (8, 6.0, 4.0, [[0, 0, 0]], True),            # one k point: a Gamma-only aliasing grid
    (24, 10.0, 6.0, [[0, 0, 0]], False),
    (48, 13.5, 12.0, [[a, b, c] for a in (0, 0.5) for b in (0, 0.5) for c in (0, 0.5)], False),
])
def test_kplan_refuses_grids_whose_pair_densities_reach_the_nyquist_plane(lib, n, L, ecut, kpts, refused):
    # the refusal is decided on the host before any CUDA call, so it is seen
    # here without a GPU; an accepted grid goes on to the device and fails
    # there (CUDA error) on this machine, or returns a plan on a GPU
    cell = cubic(L)
    reach = _pair_density_reach((n, n, n), cell, ecut, np.asarray(kpts, dtype=float))
    assert (2 * reach >= n) == refused
    kp = np.asarray(kpts, dtype=float)
    try:
        h = _lib.fock_kplan_create((n, n, n), cell, ecut, kp, np.full(len(kp), 1.0 / len(kp)), 1, (0.5,), 1)
    except _lib.FockError as e:
        assert (e.status == 3) == refused, (e.status, str(e))
        return
    _lib.fock_kplan_destroy(h)
    assert not refused
