"""torch.autograd.Function over the hand-written CUDA adjoint.

``rollout(rho0, ux0, uy0, bx0, by0, C_S, tau_nu, tau_eta, nsteps)`` runs
``nsteps`` fused LB-MHD steps from the equilibrium state of the given
fields (contiguous float64 CUDA tensors of shape (ny, nx)) and returns the
final moments (rho, ux, uy, bx, by).  Its backward is the discrete adjoint
of the step (lbmhd_adjoint_backward): checkpoints every ``every`` steps are
kept in FP64 during the forward, each segment is recomputed in the storage
format of ``precision`` and the adjoint kernel walks it backwards.
Gradients flow to the five initial fields and to C_S, tau_nu, tau_eta
(0-dim tensors).  All compute runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import lbmhd as L


class _Owned:
    """Destroys the handle when the autograd graph lets go of it."""

    def __init__(self, h):
        self.h = h

    def __del__(self):
        try:
            L.lbmhd_destroy(self.h)
        except Exception:
            pass


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, ux0, uy0, bx0, by0, C_S, tau_nu, tau_eta, nsteps, every, precision,
                params):
        ny, nx = rho0.shape
        p = L.lbmhd_params_default(precision=precision, tau_nu=float(tau_nu),
                                   tau_eta=float(tau_eta), C_S=float(C_S), **(params or {}))
        h = L.lbmhd_create(nx, ny, p)
        owned = _Owned(h)
        fields = [t.detach().contiguous() for t in (rho0, ux0, uy0, bx0, by0)]
        torch.cuda.synchronize()
        L.lbmhd_adjoint_record(h, *fields, int(nsteps), int(every))
        outs = [torch.empty_like(fields[0]) for _ in range(5)]
        L.lbmhd_moments_device(h, *outs)
        L.lbmhd_sync(h)
        ctx.owned = owned
        ctx.scalar_like = C_S
        return tuple(outs)

    @staticmethod
    def backward(ctx, g_rho, g_ux, g_uy, g_bx, g_by):
        h = ctx.owned.h
        grads = [None if g is None else g.detach().contiguous() for g in
                 (g_rho, g_ux, g_uy, g_bx, g_by)]
        torch.cuda.synchronize()
        need_fields = any(ctx.needs_input_grad[:5])
        dth, dfields = L.lbmhd_adjoint_backward(h, grads, want_fields=need_fields)
        ref = ctx.scalar_like
        th = [torch.tensor(v, dtype=torch.float64, device=ref.device) for v in dth]
        ctx.owned = None  # releases the handle
        df = dfields if dfields is not None else (None,) * 5
        return (*df, th[0], th[1], th[2], None, None, None, None)


def rollout(rho0, ux0, uy0, bx0, by0, C_S, tau_nu, tau_eta, nsteps: int, every: int = 50,
            precision: str = "fp64", params: dict | None = None):
    """Differentiable rollout; see the module docstring.  ``params``: other
    lbmhd_params fields (delta, s5..s8, les)."""
    as_t = lambda v: v if torch.is_tensor(v) else torch.tensor(float(v), dtype=torch.float64)
    return Rollout.apply(rho0, ux0, uy0, bx0, by0, as_t(C_S), as_t(tau_nu), as_t(tau_eta),
                         nsteps, every, precision, params)
