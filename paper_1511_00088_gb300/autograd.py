"""Differentiable staggered fermion action S = phi^dag (M^dag M)^{-1} phi.

The forward pass solves (4 m^2 - D_eo D_oe) X = phi with the library's CG and
evaluates S in the library (stag_action: the stationary form 2 Re<phi, X> -
Re<X, A X>, double-word FP64 sums on the GPU).  The backward pass is
hand-written in the library too (stag_action_backward): one half operator
Y = D_oe X and one pass over the links give gS times the gauge-field gradient
dS/dRe U + i dS/dIm U, and the source gradient 2 gS X.  X is kept from the
forward pass, so the backward needs no further solve.  This module only
allocates and marshals tensors.
"""
from __future__ import annotations

import torch

from . import stag


class FermionAction(torch.autograd.Function):
    """S(links, phi) for a fixed context (lattice), mass and solver settings."""

    @staticmethod
    def forward(fctx, links, phi, context, mass, tol, precision, maxiter):
        if not (links.is_cuda and phi.is_cuda):
            raise ValueError("links and phi must be CUDA tensors (complex128)")
        context.links_upload(links.detach().contiguous())
        phi_c = phi.detach().contiguous()
        xs, st, it, tr = context.cg_solve([phi_c], [mass], tol=tol, maxiter=maxiter, precision=precision)
        X = xs[0]
        S = context.action(phi_c, X, mass)
        fctx.save_for_backward(X)
        fctx.context = context
        return torch.tensor(S, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(fctx, gS):
        (X,) = fctx.saved_tensors
        g = float(gS)
        grad_links = torch.empty((4, fctx.context.V, 3, 3), dtype=torch.complex128, device=X.device) \
            if fctx.needs_input_grad[0] else None
        grad_phi = torch.empty_like(X) if fctx.needs_input_grad[1] else None
        if grad_links is not None or grad_phi is not None:
            fctx.context.action_backward(X, g, grad_links, grad_phi)
        return grad_links, grad_phi, None, None, None, None, None


def fermion_action(links, phi, context, mass, tol=1e-12, precision=stag.STAG_FP64, maxiter=100000):
    """S = phi^dag (4 m^2 - D_eo D_oe)^{-1} phi, differentiable in links and phi.

    links: (4, V, 3, 3) complex128 CUDA tensor; phi: (V/2, 3) complex128 CUDA
    tensor on the even sites; context: a stag.Context of the lattice.
    """
    return FermionAction.apply(links, phi, context, float(mass), float(tol), int(precision), int(maxiter))
