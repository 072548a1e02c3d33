"""E_x(psi, omega) as a differentiable torch function.

The exchange energy of §4 is a quartic functional of the orbitals.  Its
derivative with respect to c_j(G)* is f_j (V_x psi_j)(G), which is exactly what
``fock_apply`` returns, so the backward pass costs nothing beyond the forward:

    torch convention (gradient = 2 dL/dz* for a real loss L):
        grad_psi_G[j, G] = 2 f_j (V_x psi_j)(G) * grad_E
        grad_omega       = dE_x/domega * grad_E       (erfc kernel)

with dE_x/domega = -(Omega/2) sum_ij f_i f_j sum_G dv/domega |rho_ij(G)|^2 from
the same call.  The orbitals are Gamma-point real functions (c(-G) = c(G)*);
directional derivatives are meaningful along directions that keep that
symmetry.  The Coulomb-kernel table depends on omega, so plans are cached per
(grid, cell, cutoff, kernel, omega, precision).
"""

import numpy as np
import torch

from . import _lib
from .plan import FockPlan

_PLANS = {}


def _plan(grid, cell, ecut, kernel, omega, precision):
    key = (tuple(grid), tuple(np.asarray(cell, dtype=np.float64).ravel().tolist()), float(ecut), int(kernel),
           None if omega is None else float(omega), int(precision), torch.cuda.current_device())
    p = _PLANS.get(key)
    if p is None:
        if len(_PLANS) >= 16:
            _PLANS.pop(next(iter(_PLANS))).close()
        p = FockPlan(grid, cell, ecut, kernel, omega, precision)
        _PLANS[key] = p
    return p


class ExchangeEnergy(torch.autograd.Function):
    """forward(psi_G [nb, npw] complex128 CUDA, omega 0-d tensor, occ, plan args) -> E_x."""

    @staticmethod
    def forward(ctx, psi_G, omega, occ, grid, cell, ecut, kernel, precision):
        om = None if kernel == _lib.SPENCER_ALAVI else float(omega.detach().cpu())
        plan = _plan(grid, cell, ecut, kernel, om, precision)
        psi = psi_G.detach()
        if psi.dtype != torch.complex128:
            psi = psi.to(torch.complex128)
        psi = psi.contiguous()
        occ = np.asarray(occ, dtype=np.float64)
        vpsi, ex, dex = plan.apply(psi, occ, want_ex=True, want_dex=kernel == _lib.ERFC)
        ctx.save_for_backward(vpsi)
        ctx.occ = occ
        ctx.dex = 0.0 if dex is None else dex
        ctx.psi_dtype = psi_G.dtype
        ctx.omega_meta = (omega.device, omega.dtype)
        return torch.tensor(ex, dtype=torch.float64, device=psi_G.device)

    @staticmethod
    def backward(ctx, grad_e):
        (vpsi,) = ctx.saved_tensors
        f = torch.as_tensor(ctx.occ, dtype=torch.float64, device=vpsi.device)
        g = grad_e.to(torch.float64)
        grad_psi = None
        if ctx.needs_input_grad[0]:
            grad_psi = (2.0 * g) * (f[:, None] * vpsi)
            grad_psi = grad_psi.to(ctx.psi_dtype)
        grad_omega = None
        if ctx.needs_input_grad[1]:
            dev, dt = ctx.omega_meta
            grad_omega = (g * ctx.dex).to(device=dev, dtype=dt)
        return grad_psi, grad_omega, None, None, None, None, None, None


def exchange_energy(psi_G, occ, grid, cell, ecut, kernel=_lib.ERFC, omega=None,
                    precision=_lib.PREC_MIXED32):
    """E_x with autograd support in ``psi_G`` and (erfc kernel) ``omega``.

    ``omega`` may be a float or a 0-d tensor with ``requires_grad``.
    """
    if not torch.is_tensor(omega):
        omega = torch.tensor(0.0 if omega is None else float(omega), dtype=torch.float64)
    if isinstance(grid, int):
        grid = (grid, grid, grid)
    return ExchangeEnergy.apply(psi_G, omega, occ, tuple(grid), cell, ecut, kernel, precision)
