"""Differentiable staggered fermion action S = phi^dag (M^dag M)^{-1} phi.

The forward pass solves (4 m^2 - D_eo D_oe) X = phi with the library's CG and
returns S = Re <phi, X>.  The backward pass is hand-written: one half operator
Y = D_oe X and one pass over the links (stag_force) give the gauge-field
gradient in the torch convention dS/dRe U + i dS/dIm U; the source gradient is
2 X.  X is kept from the forward pass, so the backward needs no further solve.
All arithmetic runs in libstag (CUDA); this module only marshals tensors.
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
        xs, st, it, tr = context.cg_solve([phi.detach().contiguous()], [mass], tol=tol, maxiter=maxiter,
                                          precision=precision)
        X = xs[0]
        fctx.save_for_backward(X)
        fctx.context = context
        return torch.real(torch.vdot(phi.reshape(-1), X.reshape(-1)))

    @staticmethod
    def backward(fctx, gS):
        (X,) = fctx.saved_tensors
        grad_links = grad_phi = None
        if fctx.needs_input_grad[0]:
            G, _ = fctx.context.force(X, grad=True, lie=False)
            grad_links = gS * G
        if fctx.needs_input_grad[1]:
            grad_phi = 2.0 * gS * X
        return grad_links, grad_phi, None, None, None, None, None


def fermion_action(links, phi, context, mass, tol=1e-12, precision=stag.STAG_FP64, maxiter=100000):
    """S = phi^dag (4 m^2 - D_eo D_oe)^{-1} phi, differentiable in links and phi.

    links: (4, V, 3, 3) complex128 CUDA tensor; phi: (V/2, 3) complex128 CUDA
    tensor on the even sites; context: a stag.Context of the lattice.
    """
    return FermionAction.apply(links, phi, context, float(mass), float(tol), int(precision), int(maxiter))
