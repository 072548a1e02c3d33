"""ctypes binding of libfockx.so: the C-ABI entry points of include/fock.h under
the same names, with argument marshalling only.

Device buffers are passed as torch CUDA tensors (complex128, contiguous); the
binding hands their addresses and torch's current CUDA stream to the library.
All computation happens in the library's CUDA kernels; when the library is not
built this module raises instead of computing anything another way.
"""

import ctypes
import os

import numpy as np

SPENCER_ALAVI = 0
ERFC = 1
PREC_FP64 = 0
PREC_MIXED32 = 1
PREC_DF64 = 2
GAMMA_REAL = 1

STATUS = {
    0: "FOCK_OK",
    1: "FOCK_ERR_INVALID_ARG",
    2: "FOCK_ERR_UNSUPPORTED_SIZE",
    3: "FOCK_ERR_GRID_TOO_SMALL",
    4: "FOCK_ERR_OOM",
    5: "FOCK_ERR_CUDA",
    6: "FOCK_ERR_TIMEOUT",
}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfockx.so")

_lib = None

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)
_c_i32_p = ctypes.POINTER(ctypes.c_int32)
_c_i64_p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p

NPHASES = 6
PHASES = ("to_real", "pair_fwd", "pair_col", "pair_inv", "to_sphere", "energy")


class FockStats(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int64),
        ("phase_launches", ctypes.c_int64 * NPHASES),
        ("phase_ms", ctypes.c_double * NPHASES),
        ("chains", ctypes.c_int64),
        ("pairs", ctypes.c_int64),
        ("chain_batch", ctypes.c_int),
        ("band_batch", ctypes.c_int),
    ]


class BatchOptions(ctypes.Structure):
    _fields_ = [
        ("slot_chains", ctypes.c_int),
        ("ring", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("want_dex", ctypes.c_int),
        ("wait_limit_s", ctypes.c_double),
        ("stall_segment", ctypes.c_int),
        ("persistent", ctypes.c_int),
    ]


_SIGNATURES = {
    "fock_plan_create": [ctypes.POINTER(_vp), _c_int_p, _c_dbl_p, ctypes.c_double, ctypes.c_int,
                         _c_dbl_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint],
    "fock_gsphere": [_c_int_p, _c_dbl_p, ctypes.c_double, _c_i64_p, _c_i32_p, ctypes.c_int64],
    "fock_schedule": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_i32_p, ctypes.c_int64,
                      _c_i64_p],
    "fock_plan_set_band_block": [_vp, ctypes.c_int],
    "fock_plan_tiling_info": [_vp, ctypes.c_int, ctypes.c_int, _c_int_p, _c_int_p, _c_int_p, _c_int_p, _c_int_p],
    "fock_plan_set_tiling": [_vp, _c_int_p],
    "fock_plan_npw": [_vp, _c_i64_p],
    "fock_plan_gvectors": [_vp, _c_i32_p],
    "fock_plan_reserve": [_vp, ctypes.c_int],
    "fock_plan_set_batch": [_vp, ctypes.c_int],
    "fock_plan_device_bytes": [_vp, _c_i64_p],
    "fock_plan_columns": [_vp, _c_i64_p, _c_i64_p],
    "fock_plan_set_deterministic": [_vp, ctypes.c_int],
    "fock_plan_set_timing": [_vp, ctypes.c_int],
    "fock_plan_set_streams": [_vp, ctypes.c_int],
    "fock_plan_stats": [_vp, ctypes.POINTER(FockStats)],
    "fock_apply": [_vp, _vp, ctypes.c_int, _c_dbl_p, _vp, _c_dbl_p, _c_dbl_p, _vp],
    "fock_apply_shard": [_vp, _vp, ctypes.c_int, _c_dbl_p, ctypes.c_int, ctypes.c_int, _vp,
                         _c_dbl_p, _c_dbl_p, _vp],
    "fock_pair_energies": [_vp, _vp, ctypes.c_int, _c_i32_p, ctypes.c_int, _c_dbl_p, _c_dbl_p, _vp],
    "fock_set_occupied": [_vp, _vp, ctypes.c_int, _c_dbl_p, _vp],
    "fock_apply_fixed": [_vp, _vp, ctypes.c_int, _vp, _vp],
    "fock_pair_energies_static": [_vp, _vp, ctypes.c_int, _c_i32_p, ctypes.c_int, _c_dbl_p, _c_dbl_p,
                                  _vp],
    "fock_sternheimer_solve": [_vp, _vp, _vp, ctypes.c_int, _c_dbl_p, _vp, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, ctypes.c_int, _vp, _c_int_p, _c_dbl_p, _vp],
    "fock_batch_default_options": [ctypes.POINTER(BatchOptions)],
    "fock_batch_create": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp), _c_int_p,
                          ctypes.POINTER(_vp), ctypes.POINTER(_c_dbl_p), ctypes.POINTER(_vp),
                          ctypes.POINTER(BatchOptions)],
    "fock_batch_run": [_vp, _c_dbl_p, _c_dbl_p, _vp],
    "fock_batch_info": [_vp, _c_i64_p, _c_i64_p, _c_int_p, _c_int_p, _c_dbl_p],
    "fock_batch_last_error": [_vp],
    "fock_batch_destroy": [_vp],
    "fock_kplan_create": [ctypes.POINTER(_vp), _c_int_p, _c_dbl_p, ctypes.c_double, ctypes.c_int, _c_dbl_p,
                          _c_dbl_p, ctypes.c_int, _c_dbl_p, ctypes.c_int, ctypes.c_int],
    "fock_gsphere_k": [_c_int_p, _c_dbl_p, ctypes.c_double, _c_dbl_p, _c_i64_p, _c_i32_p, ctypes.c_int64],
    "fock_kplan_nk": [_vp, _c_int_p],
    "fock_kplan_npw": [_vp, ctypes.c_int, _c_i64_p],
    "fock_kplan_gvectors": [_vp, ctypes.c_int, _c_i32_p],
    "fock_kplan_set_batch": [_vp, ctypes.c_int],
    "fock_kplan_apply": [_vp, ctypes.POINTER(_vp), ctypes.c_int, _c_dbl_p, ctypes.POINTER(_vp), _c_dbl_p, _vp],
    "fock_kplan_last_error": [_vp],
    "fock_kplan_destroy": [_vp],
    "fock_destroy": [_vp],
    "fock_status_string": [ctypes.c_int],
    "fock_last_error": [_vp],
}


class FockError(RuntimeError):
    def __init__(self, status, message):
        self.status = int(status)
        super().__init__("%s: %s" % (STATUS.get(self.status, str(status)), message))


def load():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfockx.so is not built; run `python -m paper_1305_7313_gb300.build` "
                           "or __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = (ctypes.c_char_p if name in ("fock_status_string", "fock_last_error",
                                                   "fock_batch_last_error", "fock_kplan_last_error")
                       else ctypes.c_int)
    _lib = lib
    return lib


def _check(status, plan=None):
    if status != 0:
        msg = load().fock_last_error(plan).decode()
        raise FockError(status, msg)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _rows(t, name, npw, nrows=None):
    """Check that orbital tensor ``t`` is [nrows, npw] for the plan's sphere of
    npw plane waves, before it is touched: the library takes the row length
    from the plan, so a tensor of another sphere would be read past its end."""
    shape = tuple(getattr(t, "shape", ()))
    if len(shape) != 2 or shape[1] != npw or (nrows is not None and shape[0] != nrows):
        want = "[%s, %d]" % ("nb" if nrows is None else nrows, npw)
        raise ValueError("%s has shape %s, expected %s (the plan's sphere)" % (name, shape, want))
    return shape[0]


def _dev_ptr(t, name, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.complex128 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous complex128 tensor" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return ctypes.c_void_p(t.data_ptr())


def _dbl_array(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a, a.ctypes.data_as(_c_dbl_p)


def fock_status_string(status):
    return load().fock_status_string(int(status)).decode()


def fock_last_error(plan=None):
    return load().fock_last_error(plan).decode()


def fock_gsphere(grid, cell, ecut):
    """Miller indices [npw, 3] (int32) of the sphere in canonical order (host only)."""
    lib = load()
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    c, cp = _dbl_array(np.asarray(cell, dtype=np.float64).ravel())
    n = ctypes.c_int64()
    _check(lib.fock_gsphere(g, cp, float(ecut), ctypes.byref(n), None, 0))
    out = np.empty((n.value, 3), dtype=np.int32)
    _check(lib.fock_gsphere(g, cp, float(ecut), ctypes.byref(n), out.ctypes.data_as(_c_i32_p), n.value))
    return out


def fock_schedule(nb, shard=0, nshards=1, band_block=0):
    """Unique pairs [npairs, 2] (int32) that shard `shard` of `nshards` evaluates (host only)."""
    lib = load()
    n = ctypes.c_int64()
    _check(lib.fock_schedule(int(nb), int(band_block), int(shard), int(nshards), None, 0, ctypes.byref(n)))
    out = np.empty((n.value, 2), dtype=np.int32)
    _check(lib.fock_schedule(int(nb), int(band_block), int(shard), int(nshards),
                             out.ctypes.data_as(_c_i32_p), n.value, ctypes.byref(n)))
    return out


def fock_plan_set_band_block(plan, band_block):
    _check(load().fock_plan_set_band_block(plan, int(band_block)), plan)


def fock_plan_create(grid, cell, ecut, kind=SPENCER_ALAVI, kparams=(), prec=PREC_FP64, flags=GAMMA_REAL):
    """Create a plan; returns its handle (an int)."""
    lib = load()
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    c, cp = _dbl_array(np.asarray(cell, dtype=np.float64).ravel())
    kp, kpp = _dbl_array(list(kparams) if len(kparams) else [0.0])
    h = ctypes.c_void_p()
    _check(lib.fock_plan_create(ctypes.byref(h), g, cp, float(ecut), int(kind), kpp, len(kparams),
                                int(prec), int(flags)))
    return h.value


def fock_plan_npw(plan):
    n = ctypes.c_int64()
    _check(load().fock_plan_npw(plan, ctypes.byref(n)), plan)
    return n.value


def fock_plan_gvectors(plan):
    out = np.empty((fock_plan_npw(plan), 3), dtype=np.int32)
    _check(load().fock_plan_gvectors(plan, out.ctypes.data_as(_c_i32_p)), plan)
    return out


def fock_plan_reserve(plan, nb_max):
    _check(load().fock_plan_reserve(plan, int(nb_max)), plan)


def fock_plan_set_batch(plan, chain_batch):
    _check(load().fock_plan_set_batch(plan, int(chain_batch)), plan)


def fock_plan_set_timing(plan, enable):
    _check(load().fock_plan_set_timing(plan, 1 if enable else 0), plan)


def fock_plan_stats(plan):
    """Counters of the last call as a dict (per-phase device times need timing on)."""
    s = FockStats()
    _check(load().fock_plan_stats(plan, ctypes.byref(s)), plan)
    return {
        "launches": s.launches,
        "phase_launches": dict(zip(PHASES, list(s.phase_launches))),
        "phase_ms": dict(zip(PHASES, list(s.phase_ms))),
        "chains": s.chains,
        "pairs": s.pairs,
        "chain_batch": s.chain_batch,
        "band_batch": s.band_batch,
    }


PASSES = ("pair_fwd", "pair_col", "pair_inv")


def fock_plan_tiling_info(plan, pass_, tile):
    """Radix plan of tiling `tile` of pair pass `pass_` (0 fwd, 1 col, 2 inv):
    dict(radices, threads_per_line, threads, ntiles)."""
    r = (ctypes.c_int * 8)()
    nst, tl, thr, nt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().fock_plan_tiling_info(plan, int(pass_), int(tile), r, ctypes.byref(nst), ctypes.byref(tl),
                                        ctypes.byref(thr), ctypes.byref(nt)), plan)
    return {"radices": list(r[:nst.value]), "threads_per_line": tl.value, "threads": thr.value,
            "ntiles": nt.value}


def fock_plan_set_tiling(plan, tiles):
    """Tiling (0 or 1) of the forward plane, column and inverse plane passes."""
    t = (ctypes.c_int * 3)(*[int(x) for x in tiles])
    _check(load().fock_plan_set_tiling(plan, t), plan)


def fock_plan_set_streams(plan, streams):
    """Streams (1 to 4) the pair-pass launches of an apply rotate over."""
    _check(load().fock_plan_set_streams(plan, int(streams)), plan)


def fock_plan_device_bytes(plan):
    n = ctypes.c_int64()
    _check(load().fock_plan_device_bytes(plan, ctypes.byref(n)), plan)
    return n.value


def fock_plan_set_deterministic(plan, enable=True):
    """Exact fixed-point accumulation and fixed-order energy sums (FP64 and double-float plans)."""
    _check(load().fock_plan_set_deterministic(plan, 1 if enable else 0), plan)


def fock_plan_columns(plan):
    """(kept, total) columns of the stored half spectrum the column pass transforms."""
    k = ctypes.c_int64()
    t = ctypes.c_int64()
    _check(load().fock_plan_columns(plan, ctypes.byref(k), ctypes.byref(t)), plan)
    return k.value, t.value


def fock_apply(plan, psi_G, occ, vpsi_G, want_ex=True, want_dex=False, stream=None):
    """V_x psi into ``vpsi_G``; returns (E_x or None, dE_x/domega or None)."""
    npw = fock_plan_npw(plan)
    nb = _rows(psi_G, "psi_G", npw)
    _rows(vpsi_G, "vpsi_G", npw, nb)
    a = _dev_ptr(psi_G, "psi_G")
    b = _dev_ptr(vpsi_G, "vpsi_G", (nb, npw))
    o, op = _dbl_array(occ)
    if o.shape != (nb,):
        raise ValueError("occ must have one entry per band")
    ex, dex = ctypes.c_double(), ctypes.c_double()
    _check(load().fock_apply(plan, a, nb, op, b, ctypes.byref(ex) if want_ex else None,
                             ctypes.byref(dex) if want_dex else None, _stream(stream)), plan)
    return (ex.value if want_ex else None), (dex.value if want_dex else None)


def fock_apply_shard(plan, psi_G, occ, shard, nshards, vpsi_G, want_ex=True, want_dex=False, stream=None):
    """Part ``shard`` of ``nshards`` of the pair loop; returns the partial (E_x, dE_x/domega)."""
    npw = fock_plan_npw(plan)
    nb = _rows(psi_G, "psi_G", npw)
    _rows(vpsi_G, "vpsi_G", npw, nb)
    a = _dev_ptr(psi_G, "psi_G")
    b = _dev_ptr(vpsi_G, "vpsi_G", (nb, npw))
    o, op = _dbl_array(occ)
    ex, dex = ctypes.c_double(), ctypes.c_double()
    _check(load().fock_apply_shard(plan, a, nb, op, int(shard), int(nshards), b,
                                   ctypes.byref(ex) if want_ex else None,
                                   ctypes.byref(dex) if want_dex else None, _stream(stream)), plan)
    return (ex.value if want_ex else None), (dex.value if want_dex else None)


def fock_set_occupied(plan, psi_G, occ, stream=None):
    """Fix the occupied orbitals (device [nb, npw] complex128) that define V_x."""
    nb = _rows(psi_G, "psi_G", fock_plan_npw(plan))
    a = _dev_ptr(psi_G, "psi_G")
    o, op = _dbl_array(occ)
    if o.shape != (nb,):
        raise ValueError("occ must have one entry per band")
    _check(load().fock_set_occupied(plan, a, nb, op, _stream(stream)), plan)


def fock_apply_fixed(plan, phi_G, vphi_G, stream=None):
    """V_x phi for trial orbitals with the V_x fixed by fock_set_occupied."""
    npw = fock_plan_npw(plan)
    nt = _rows(phi_G, "phi_G", npw)
    _rows(vphi_G, "vphi_G", npw, nt)
    a = _dev_ptr(phi_G, "phi_G")
    b = _dev_ptr(vphi_G, "vphi_G", (nt, npw))
    _check(load().fock_apply_fixed(plan, a, nt, b, _stream(stream)), plan)


def fock_pair_energies(plan, psi_G, pairs, want_d=False, stream=None):
    """e_ij (and d_ij) for the listed (i, j) pairs; numpy float64 arrays."""
    nb = _rows(psi_G, "psi_G", fock_plan_npw(plan))
    a = _dev_ptr(psi_G, "psi_G")
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    e = np.empty(len(pr))
    d = np.empty(len(pr))
    _check(load().fock_pair_energies(plan, a, nb, pr.ctypes.data_as(_c_i32_p), len(pr),
                                     e.ctypes.data_as(_c_dbl_p),
                                     d.ctypes.data_as(_c_dbl_p) if want_d else None,
                                     _stream(stream)), plan)
    return (e, d) if want_d else e


def fock_pair_energies_static(plan, psi_G, pairs, want_d=False, stream=None):
    """fock_pair_energies computed in the library's static device scratch (no allocation)."""
    nb = _rows(psi_G, "psi_G", fock_plan_npw(plan))
    a = _dev_ptr(psi_G, "psi_G")
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    e = np.empty(len(pr))
    d = np.empty(len(pr))
    _check(load().fock_pair_energies_static(plan, a, nb, pr.ctypes.data_as(_c_i32_p), len(pr),
                                            e.ctypes.data_as(_c_dbl_p),
                                            d.ctypes.data_as(_c_dbl_p) if want_d else None,
                                            _stream(stream)), plan)
    return (e, d) if want_d else e


def fock_sternheimer_solve(plan, ntot, vloc, u_G, eps, w_G, alpha, tol, maxiter=1000, g_G=None, stream=None):
    """(g, iters, resid): CG solution of (H - eps_n + alpha P) g_n = -Q w_n for
    H = kinetic + V(r) on the plan's sphere.  ``ntot``: the plan's grid points
    N^3; ``vloc``: contiguous CUDA float64 tensor with ntot elements;
    ``u_G`` / ``w_G``: CUDA complex128 [nocc / nrhs, npw]; ``eps``: host [nrhs]."""
    import torch
    npw = fock_plan_npw(plan)
    nocc = _rows(u_G, "u_G", npw)
    nrhs = _rows(w_G, "w_G", npw)
    if not (isinstance(vloc, torch.Tensor) and vloc.is_cuda and vloc.dtype == torch.float64
            and vloc.is_contiguous()):
        raise TypeError("vloc must be a contiguous CUDA float64 tensor")
    if vloc.numel() != int(ntot):
        raise ValueError("vloc has %d values, the plan's grid %d" % (vloc.numel(), int(ntot)))
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).ravel())
    if eps.shape != (nrhs,):
        raise ValueError("eps must hold one value per right-hand ket (%d)" % nrhs)
    if g_G is None:
        g_G = torch.empty_like(w_G)
    iters = (ctypes.c_int * nrhs)()
    resid = (ctypes.c_double * nrhs)()
    _check(load().fock_sternheimer_solve(plan, ctypes.c_void_p(vloc.data_ptr()), _dev_ptr(u_G, "u_G"), nocc,
                                         eps.ctypes.data_as(_c_dbl_p), _dev_ptr(w_G, "w_G"), nrhs,
                                         float(alpha), float(tol), int(maxiter),
                                         _dev_ptr(g_G, "g_G", tuple(w_G.shape)), iters, resid,
                                         _stream(stream)), plan)
    return g_G, np.array(iters[:], dtype=np.int64), np.array(resid[:])


def _check_batch(status, batch=None):
    if status != 0:
        raise FockError(status, load().fock_batch_last_error(batch).decode())


def fock_batch_default_options():
    o = BatchOptions()
    _check_batch(load().fock_batch_default_options(ctypes.byref(o)))
    return {f: getattr(o, f) for f, _ in BatchOptions._fields_}


def fock_batch_create(plans, psi_G, occ, vpsi_G, **options):
    """Batch handle for systems (plan handles, device psi/vpsi tensors, host occupations)."""
    n = len(plans)
    o = BatchOptions()
    _check_batch(load().fock_batch_default_options(ctypes.byref(o)))
    for k, v in options.items():
        setattr(o, k, v)
    if not (len(psi_G) == len(vpsi_G) == len(occ) == n):
        raise ValueError("one psi_G, vpsi_G and occ per plan")
    rows = []
    for k, (pl, p, v) in enumerate(zip(plans, psi_G, vpsi_G)):
        npw = fock_plan_npw(pl)
        rows.append(_rows(p, "psi_G[%d]" % k, npw))
        _rows(v, "vpsi_G[%d]" % k, npw, rows[-1])
    ph = (_vp * n)(*plans)
    nb = (ctypes.c_int * n)(*rows)
    pp = (_vp * n)(*[_dev_ptr(p, "psi_G").value for p in psi_G])
    vp = (_vp * n)(*[_dev_ptr(v, "vpsi_G", tuple(p.shape)).value for v, p in zip(vpsi_G, psi_G)])
    occ_arrays = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in occ]
    op = (_c_dbl_p * n)(*[a.ctypes.data_as(_c_dbl_p) for a in occ_arrays])
    h = _vp()
    _check_batch(load().fock_batch_create(ctypes.byref(h), n, ph, nb, pp, op, vp, ctypes.byref(o)))
    return h.value


def fock_batch_run(batch, nsys, stream=None):
    """Run the batch; returns (E_x[nsys], dE_x/domega[nsys]) as numpy arrays."""
    ex = np.empty(nsys)
    dex = np.empty(nsys)
    _check_batch(load().fock_batch_run(batch, ex.ctypes.data_as(_c_dbl_p), dex.ctypes.data_as(_c_dbl_p),
                                       _stream(stream)), batch)
    return ex, dex


def fock_batch_info(batch):
    la, ta = ctypes.c_int64(), ctypes.c_int64()
    gr, sg = ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    _check_batch(load().fock_batch_info(batch, ctypes.byref(la), ctypes.byref(ta), ctypes.byref(gr),
                                        ctypes.byref(sg), ctypes.byref(ms)), batch)
    return {"launches": la.value, "tasks": ta.value, "grid": gr.value, "segments": sg.value,
            "persist_ms": ms.value}


def fock_batch_last_error(batch=None):
    return load().fock_batch_last_error(batch).decode()


def fock_batch_destroy(batch):
    _check_batch(load().fock_batch_destroy(batch))


def _check_k(status, plan=None):
    if status != 0:
        raise FockError(status, load().fock_kplan_last_error(plan).decode())


def fock_kplan_create(grid, cell, ecut, kpts, weights, kind=SPENCER_ALAVI, kparams=(), prec=PREC_FP64):
    lib = load()
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    c, cp = _dbl_array(np.asarray(cell, dtype=np.float64).ravel())
    k, kp = _dbl_array(np.asarray(kpts, dtype=np.float64).reshape(-1, 3).ravel())
    w, wp = _dbl_array(np.asarray(weights, dtype=np.float64).ravel())
    pr, prp = _dbl_array(list(kparams) if len(kparams) else [0.0])
    h = _vp()
    _check_k(lib.fock_kplan_create(ctypes.byref(h), g, cp, float(ecut), len(w), kp, wp, int(kind), prp,
                                   len(kparams), int(prec)))
    return h.value


def fock_gsphere_k(grid, cell, ecut, kpt):
    """Miller indices [npw, 3] of S_k in canonical order (host only)."""
    lib = load()
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    c, cp = _dbl_array(np.asarray(cell, dtype=np.float64).ravel())
    k, kp = _dbl_array(np.asarray(kpt, dtype=np.float64).ravel())
    n = ctypes.c_int64()
    _check_k(lib.fock_gsphere_k(g, cp, float(ecut), kp, ctypes.byref(n), None, 0))
    out = np.empty((n.value, 3), dtype=np.int32)
    _check_k(lib.fock_gsphere_k(g, cp, float(ecut), kp, ctypes.byref(n), out.ctypes.data_as(_c_i32_p), n.value))
    return out


def fock_kplan_nk(plan):
    """Number of k points of the plan."""
    n = ctypes.c_int()
    _check_k(load().fock_kplan_nk(plan, ctypes.byref(n)), plan)
    return n.value


def fock_kplan_npw(plan, k):
    """Number of plane waves of k point ``k``."""
    n = ctypes.c_int64()
    _check_k(load().fock_kplan_npw(plan, int(k), ctypes.byref(n)), plan)
    return n.value


def fock_kplan_gvectors(plan, k):
    n = ctypes.c_int64()
    _check_k(load().fock_kplan_npw(plan, int(k), ctypes.byref(n)), plan)
    out = np.empty((n.value, 3), dtype=np.int32)
    _check_k(load().fock_kplan_gvectors(plan, int(k), out.ctypes.data_as(_c_i32_p)), plan)
    return out


def fock_kplan_set_batch(plan, chain_batch):
    _check_k(load().fock_kplan_set_batch(plan, int(chain_batch)), plan)


def fock_kplan_apply(plan, psi_G, occ, vpsi_G, want_ex=True, stream=None):
    """V_x psi for every k (lists of device tensors [nb, npw_k]); returns E_x or None.

    The library reads one psi_G / vpsi_G pointer and one row of ``occ`` per k
    point of the plan, so the list lengths and the occupation shape are checked
    against the plan's k-point count before any pointer is formed."""
    nk = fock_kplan_nk(plan)
    if len(psi_G) != nk or len(vpsi_G) != nk:
        raise ValueError("the plan has %d k points: got %d psi_G and %d vpsi_G tensors"
                         % (nk, len(psi_G), len(vpsi_G)))
    nb = None
    for k in range(nk):
        npw = fock_kplan_npw(plan, k)
        nb = _rows(psi_G[k], "psi_G[%d]" % k, npw, nb)  # every k point holds the same bands
        _rows(vpsi_G[k], "vpsi_G[%d]" % k, npw, nb)
    occ = np.asarray(occ, dtype=np.float64)
    if occ.shape != (nk, nb):
        raise ValueError("occ has shape %s, expected (%d, %d): one row of occupations per k point"
                         % (occ.shape, nk, nb))
    pp = (_vp * nk)(*[_dev_ptr(p, "psi_G").value for p in psi_G])
    vp = (_vp * nk)(*[_dev_ptr(v, "vpsi_G", tuple(p.shape)).value for v, p in zip(vpsi_G, psi_G)])
    o, op = _dbl_array(occ.ravel())
    ex = ctypes.c_double()
    _check_k(load().fock_kplan_apply(plan, pp, nb, op, vp, ctypes.byref(ex) if want_ex else None,
                                     _stream(stream)), plan)
    return ex.value if want_ex else None


def fock_kplan_destroy(plan):
    _check_k(load().fock_kplan_destroy(plan))


def fock_destroy(plan):
    _check(load().fock_destroy(plan))
