"""torch.autograd.Function for the pseudofermion action of the red/black
Moebius operator: S = phi^dag (M^dag M)^-1 phi as a function of the links U
and of (b5, c5). The forward pass solves once for S; the backward pass calls
mdwf_force, which solves again for X = (M^dag M)^-1 phi (the solution is
recomputed, not kept between the passes) and returns dS/dU and dS/d(b5, c5).
Gradients follow torch's convention for complex inputs: dS/dRe U + i dS/dIm U.

b5c5 holds either the constant pair (b5, c5), shape (2,), or per-slice
coefficients (Sec. 2.1, Eq. DWaction), shape (2, Ls): row 0 is b5(s), row 1 is
c5(s); its gradient has the same shape. A chemical potential mu (Sec. 6.6)
multiplies the forward time links by e^{+mu} and the backward ones by e^{-mu};
it is a fixed parameter, not differentiated.
"""
from __future__ import annotations

import torch

import numpy as np

from . import (MDWF_F64, mdwf_create, mdwf_destroy, mdwf_force, mdwf_load_gauge,
               mdwf_set_chemical_potential, mdwf_set_s_coefficients)


def _open(U, b5c5, dims, Ls, M5, mf, mu):
    """A library context for these parameters with the links loaded."""
    bc = b5c5.detach().cpu().double().numpy()
    if bc.shape not in ((2,), (2, Ls)):
        raise ValueError(f"b5c5 must have shape (2,) or (2, {Ls}), not {tuple(bc.shape)}")
    per_slice = bc.ndim == 2
    b5, c5 = (float(bc[0, 0]), float(bc[1, 0])) if per_slice else (float(bc[0]), float(bc[1]))
    h = mdwf_create(dims, Ls, M5, b5, c5, mf)
    try:
        if per_slice:
            mdwf_set_s_coefficients(h, bc[0], bc[1])
        if mu:
            mdwf_set_chemical_potential(h, mu)
        mdwf_load_gauge(h, U.detach().contiguous())
    except BaseException:
        mdwf_destroy(h)
        raise
    return h


class MobiusAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, b5c5, phi, dims, Ls, M5, mf, tol=1e-12, inner_prec=MDWF_F64, mu=0.0):
        """U: complex128 (T, Z, Y, X, 4, 3, 3) on cuda; b5c5: float64 (2,) or (2, Ls); phi: complex128
        odd field (Ls, V/2, 4, 3) on cuda. Returns S as a 0-d float64 tensor."""
        h = _open(U, b5c5, dims, Ls, M5, mf, mu)
        try:
            S, _, _, _, _ = mdwf_force(h, None, phi.detach().contiguous(), tol=tol, inner_prec=inner_prec)
        finally:
            mdwf_destroy(h)
        ctx.save_for_backward(U, b5c5, phi)
        ctx.params = (tuple(dims), int(Ls), float(M5), float(mf), float(tol), int(inner_prec), float(mu))
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gS):
        U, b5c5, phi = ctx.saved_tensors
        dims, Ls, M5, mf, tol, inner_prec, mu = ctx.params
        h = _open(U, b5c5, dims, Ls, M5, mf, mu)
        try:
            G = torch.empty_like(U)
            _, db5, dc5, _, _ = mdwf_force(h, G, phi.detach().contiguous(), tol=tol, inner_prec=inner_prec)
        finally:
            mdwf_destroy(h)
        gU = G * gS if ctx.needs_input_grad[0] else None
        gb = None
        if ctx.needs_input_grad[1]:
            d = np.stack([np.atleast_1d(db5), np.atleast_1d(dc5)]).reshape(b5c5.shape)
            gb = torch.tensor(d, dtype=torch.float64, device=b5c5.device) * gS
        return gU, gb, None, None, None, None, None, None, None, None


def mobius_action(U, b5c5, phi, dims, Ls, M5, mf, tol=1e-12, inner_prec=MDWF_F64, mu=0.0):
    return MobiusAction.apply(U, b5c5, phi, dims, Ls, M5, mf, tol, inner_prec, mu)
