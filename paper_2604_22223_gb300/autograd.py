"""torch.autograd wrappers of one GW iteration (qa_gw_step / qa_gw_backward)
and of the GW grand potential (qa_free_energy / qa_free_energy_backward).

    step = GWStep.apply(G_in, t, V, ctx)           -> (G_out, Sigma^C(k, tau), n_local)
    omega = FreeEnergy.apply(G_in, t, V, ctx, mu, M) -> Omega[G_in] (scalar)

`t` and `V` are complex128 CPU tensors holding the context's hopping and
interaction values (the same arrays as the model); they carry the gradients
dL/dRe + i dL/dIm returned by the hand-written adjoint.  The chemical
potential of each forward step is held fixed in the backward pass, and
unrolled iterations checkpoint only their input G and mu (the adjoint
recomputes P and W from G).
"""
from __future__ import annotations

import numpy as np
import torch

from . import qa


class GWStep(torch.autograd.Function):
    @staticmethod
    def forward(fctx, G_in, t, V, ctx):
        G_out, mu, n, _ = ctx.step(G_in)
        sig = ctx.get(qa.QA_SIGC_KTAU)
        fctx.ctx = ctx
        fctx.mu = mu
        fctx.save_for_backward(G_in)
        return G_out, sig, torch.from_numpy(n.copy())

    @staticmethod
    def backward(fctx, gG, gS, gn):
        (G_in,) = fctx.saved_tensors
        ctx = fctx.ctx
        nbar = None if gn is None else gn.detach().cpu().numpy()
        Gb, gt, gV = ctx.backward(G_in.contiguous(), fctx.mu,
                                  None if gG is None else gG.contiguous(),
                                  None if gS is None else gS.contiguous(), nbar)
        return Gb, torch.from_numpy(gt), torch.from_numpy(gV), None


class FreeEnergy(torch.autograd.Function):
    """Omega[G] of qa_free_energy as a differentiable scalar of G, t(R) and V(R)
    (the values of t and V are the context's; the tensors carry the gradients)."""

    @staticmethod
    def forward(fctx, G_in, t, V, ctx, mu, M):
        om, _ = ctx.free_energy(G_in, mu, M)
        fctx.ctx, fctx.mu, fctx.M = ctx, mu, M
        fctx.save_for_backward(G_in)
        return torch.tensor(om, dtype=torch.float64)

    @staticmethod
    def backward(fctx, gO):
        (G_in,) = fctx.saved_tensors
        Gb, gt, gV = fctx.ctx.free_energy_backward(G_in.contiguous(), fctx.mu, fctx.M, float(gO))
        return Gb, torch.from_numpy(gt), torch.from_numpy(gV), None, None, None


def unrolled(ctx, t, V, n_iter, G0=None):
    """n_iter checkpointed iterations from G0 (default: the context's G0)."""
    G = ctx.get(qa.QA_G0) if G0 is None else G0
    outs = []
    for _ in range(n_iter):
        G, sig, n = GWStep.apply(G, t, V, ctx)
        outs.append((G, sig, n))
    return outs
