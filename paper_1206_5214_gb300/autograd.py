"""torch.autograd.Function for the pseudofermion action of the red/black
Moebius operator: S = phi^dag (M^dag M)^-1 phi as a function of the links U
and of (b5, c5). The forward pass solves once for S; the backward pass calls
mdwf_force, which solves again for X = (M^dag M)^-1 phi (the solution is
recomputed, not kept between the passes) and returns dS/dU and dS/d(b5, c5).
Gradients follow torch's convention for complex inputs: dS/dRe U + i dS/dIm U.
"""
from __future__ import annotations

import torch

from . import MDWF_F64, mdwf_create, mdwf_destroy, mdwf_force, mdwf_load_gauge


class MobiusAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, b5c5, phi, dims, Ls, M5, mf, tol=1e-12, inner_prec=MDWF_F64):
        """U: complex128 (T, Z, Y, X, 4, 3, 3) on cuda; b5c5: float64 (2,); phi: complex128 odd field
        (Ls, V/2, 4, 3) on cuda. Returns S as a 0-d float64 tensor."""
        b5, c5 = (float(v) for v in b5c5.detach().cpu())
        h = mdwf_create(dims, Ls, M5, b5, c5, mf)
        try:
            mdwf_load_gauge(h, U.detach().contiguous())
            S, _, _, _, _ = mdwf_force(h, None, phi.detach().contiguous(), tol=tol, inner_prec=inner_prec)
        finally:
            mdwf_destroy(h)
        ctx.save_for_backward(U, b5c5, phi)
        ctx.params = (tuple(dims), int(Ls), float(M5), float(mf), float(tol), int(inner_prec))
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gS):
        U, b5c5, phi = ctx.saved_tensors
        dims, Ls, M5, mf, tol, inner_prec = ctx.params
        b5, c5 = (float(v) for v in b5c5.detach().cpu())
        h = mdwf_create(dims, Ls, M5, b5, c5, mf)
        try:
            mdwf_load_gauge(h, U.detach().contiguous())
            G = torch.empty_like(U)
            _, db5, dc5, _, _ = mdwf_force(h, G, phi.detach().contiguous(), tol=tol, inner_prec=inner_prec)
        finally:
            mdwf_destroy(h)
        gU = G * gS if ctx.needs_input_grad[0] else None
        gb = (torch.tensor([db5, dc5], dtype=torch.float64, device=b5c5.device) * gS
              if ctx.needs_input_grad[1] else None)
        return gU, gb, None, None, None, None, None, None, None


def mobius_action(U, b5c5, phi, dims, Ls, M5, mf, tol=1e-12, inner_prec=MDWF_F64):
    return MobiusAction.apply(U, b5c5, phi, dims, Ls, M5, mf, tol, inner_prec)
