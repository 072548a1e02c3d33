"""Object wrapper around one fock_plan_t (the plan of include/fock.h)."""

import numpy as np

from . import _lib


class FockPlan:
    """A plane-wave cell on an N^3 grid with one Coulomb kernel and precision.

    ``kernel``: ``SPENCER_ALAVI`` or ``ERFC`` (then ``omega`` in bohr^-1);
    ``precision``: ``PREC_FP64``, ``PREC_MIXED32`` or ``PREC_DF64`` (double-float).
    """

    def __init__(self, grid, cell, ecut, kernel=_lib.SPENCER_ALAVI, omega=None,
                 precision=_lib.PREC_FP64):
        if isinstance(grid, int):
            grid = (grid, grid, grid)
        kp = () if kernel == _lib.SPENCER_ALAVI else (float(omega),)
        self.grid = tuple(int(g) for g in grid)
        self.cell = np.asarray(cell, dtype=np.float64).reshape(3, 3)
        self.ecut = float(ecut)
        self.kernel = kernel
        self.omega = omega
        self.precision = precision
        self.handle = None
        self.handle = _lib.fock_plan_create(self.grid, self.cell, self.ecut, kernel, kp, precision)
        self.npw = _lib.fock_plan_npw(self.handle)
        self._miller = None

    @property
    def miller(self):
        if self._miller is None:
            self._miller = _lib.fock_plan_gvectors(self.handle)
        return self._miller

    @property
    def volume(self):
        return float(abs(np.linalg.det(self.cell)))

    def set_batch(self, chain_batch):
        _lib.fock_plan_set_batch(self.handle, chain_batch)

    def set_band_block(self, band_block):
        _lib.fock_plan_set_band_block(self.handle, band_block)

    def set_streams(self, streams):
        """1 to 4 streams for the pair-pass launches (more than 1: neighbouring launches overlap)."""
        _lib.fock_plan_set_streams(self.handle, streams)

    def set_timing(self, enable):
        _lib.fock_plan_set_timing(self.handle, enable)

    def stats(self):
        return _lib.fock_plan_stats(self.handle)

    def reserve(self, nb_max):
        _lib.fock_plan_reserve(self.handle, nb_max)

    def tilings(self):
        """Per pair pass, the list of its FFT tilings (radix plans) as dicts."""
        out = {}
        for p, name in enumerate(_lib.PASSES):
            first = _lib.fock_plan_tiling_info(self.handle, p, 0)
            out[name] = [first] + [_lib.fock_plan_tiling_info(self.handle, p, t) for t in range(1, first["ntiles"])]
        return out

    def set_tiling(self, tiles):
        """Tiling index (0 or 1) of the forward plane, column and inverse plane passes."""
        _lib.fock_plan_set_tiling(self.handle, tiles)

    def device_bytes(self):
        return _lib.fock_plan_device_bytes(self.handle)

    def set_deterministic(self, enable=True):
        """Bitwise reproducible results: exact fixed-point V_x psi sums, fixed-order energies."""
        _lib.fock_plan_set_deterministic(self.handle, enable)

    def columns(self):
        """(kept, total) half-spectrum columns the column pass transforms."""
        return _lib.fock_plan_columns(self.handle)

    def apply(self, psi_G, occ, vpsi_G=None, want_ex=True, want_dex=False, stream=None):
        """(V_x psi, E_x, dE_x/domega) for device orbitals ``psi_G`` [nb, npw] complex128."""
        import torch
        if vpsi_G is None:
            vpsi_G = torch.empty_like(psi_G)
        ex, dex = _lib.fock_apply(self.handle, psi_G, occ, vpsi_G, want_ex, want_dex, stream)
        return vpsi_G, ex, dex

    def set_occupied(self, psi_G, occ, stream=None):
        """Fix the occupied set that defines V_x (kept in real space in the plan)."""
        _lib.fock_set_occupied(self.handle, psi_G, occ, stream)

    def apply_fixed(self, phi_G, vphi_G=None, stream=None):
        """V_x phi for trial orbitals with the operator fixed by :meth:`set_occupied`."""
        import torch
        if vphi_G is None:
            vphi_G = torch.empty_like(phi_G)
        _lib.fock_apply_fixed(self.handle, phi_G, vphi_G, stream)
        return vphi_G

    def apply_shard(self, psi_G, occ, shard, nshards, vpsi_G=None, want_ex=True, want_dex=False,
                    stream=None):
        import torch
        if vpsi_G is None:
            vpsi_G = torch.empty_like(psi_G)
        ex, dex = _lib.fock_apply_shard(self.handle, psi_G, occ, shard, nshards, vpsi_G, want_ex,
                                        want_dex, stream)
        return vpsi_G, ex, dex

    def apply_host(self, psi_host, occ, out_host=None, want_dex=False):
        """End-to-end call from host memory: copy in, apply, copy the result back.

        ``psi_host`` is a (preferably pinned) CPU complex128 tensor or a numpy
        array; returns (V_x psi on the host, E_x, dE_x/domega).
        """
        import torch
        if isinstance(psi_host, np.ndarray):
            psi_host = torch.from_numpy(np.ascontiguousarray(psi_host))
        dev = torch.device("cuda", torch.cuda.current_device())
        psi = psi_host.to(dev, non_blocking=True)
        vpsi = torch.empty_like(psi)
        ex, dex = _lib.fock_apply(self.handle, psi, occ, vpsi, True, want_dex)
        if out_host is None:
            out_host = torch.empty(vpsi.shape, dtype=vpsi.dtype, pin_memory=True)
        out_host.copy_(vpsi, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return out_host, ex, dex

    def pair_energies(self, psi_G, pairs, want_d=False, stream=None):
        return _lib.fock_pair_energies(self.handle, psi_G, pairs, want_d, stream)

    def sternheimer(self, vloc, u_G, eps, w_G, alpha, tol, maxiter=1000, g_G=None, stream=None):
        """(g, iters, resid) solving (H - eps_n + alpha P) g_n = -Q w_n for the
        model H = kinetic + V(r) on this plan's sphere (FP64 plans): the
        Sternheimer equation of §3.1 by CG with converged/unconverged band
        regrouping.  ``vloc``: CUDA float64 [N, N, N]; ``u_G``: occupied
        states, ``w_G``: right-hand kets, CUDA complex128 [*, npw]."""
        ntot = self.grid[0] * self.grid[1] * self.grid[2]
        return _lib.fock_sternheimer_solve(self.handle, ntot, vloc, u_G, eps, w_G, alpha, tol, maxiter, g_G, stream)

    def close(self):
        if self.handle is not None:
            _lib.fock_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class FockBatch:
    """Many systems in one batched apply, replayed as one CUDA graph; the pair
    passes run as one graph branch per system, one persistent launch or one
    dataflow launch (option ``persistent`` = 0, 1, 2).  ``plans``: distinct :class:`FockPlan` objects of one
    precision; ``psi``: device complex128 tensors [nb_s, npw_s]; ``occ``: host
    occupations.  Output tensors are allocated here and kept: every
    :meth:`run` overwrites ``self.vpsi``.  Options as in ``fock_batch_options``.
    """

    def __init__(self, plans, psi, occ, **options):
        import torch
        self.plans = list(plans)
        self.psi = list(psi)
        self.occ = [np.asarray(o, dtype=np.float64).copy() for o in occ]
        self.vpsi = [torch.empty_like(p) for p in self.psi]
        self.handle = None
        self.handle = _lib.fock_batch_create([p.handle for p in self.plans], self.psi, self.occ, self.vpsi,
                                             **options)

    def run(self, stream=None):
        """(E_x per system, dE_x/domega per system); V_x psi lands in self.vpsi."""
        return _lib.fock_batch_run(self.handle, len(self.plans), stream)

    def info(self):
        return _lib.fock_batch_info(self.handle)

    def close(self):
        if self.handle is not None:
            _lib.fock_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FockKPlan:
    """Brillouin-zone-sampled cell: ``kpts`` [nk, 3] in reduced coordinates with
    ``weights`` [nk]; one plane-wave sphere per k point (``miller(k)``)."""

    def __init__(self, grid, cell, ecut, kpts, weights, kernel=_lib.SPENCER_ALAVI, omega=None,
                 precision=_lib.PREC_FP64):
        if isinstance(grid, int):
            grid = (grid, grid, grid)
        kp = () if kernel == _lib.SPENCER_ALAVI else (float(omega),)
        self.grid = tuple(int(g) for g in grid)
        self.kpts = np.asarray(kpts, dtype=np.float64).reshape(-1, 3)
        self.weights = np.asarray(weights, dtype=np.float64).ravel()
        self.handle = None
        self.handle = _lib.fock_kplan_create(self.grid, cell, ecut, self.kpts, self.weights, kernel, kp, precision)
        self._miller = {}

    def miller(self, k):
        if k not in self._miller:
            self._miller[k] = _lib.fock_kplan_gvectors(self.handle, k)
        return self._miller[k]

    def set_batch(self, chain_batch):
        _lib.fock_kplan_set_batch(self.handle, chain_batch)

    def apply(self, psi, occ, stream=None):
        """(list of V_x psi tensors, E_x) for device orbitals ``psi`` (one tensor per k)."""
        import torch
        out = [torch.empty_like(p) for p in psi]
        ex = _lib.fock_kplan_apply(self.handle, psi, occ, out, True, stream)
        return out, ex

    def close(self):
        if self.handle is not None:
            _lib.fock_kplan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
