"""torch.autograd bindings of the differentiable part of the path.

The discrete decisions (solid mask, refine flags, which links exist, which
triangle each link crosses) carry no gradient.  q is differentiable with respect
to the vertex positions through the crossed triangle (emb_cutlinks_backward),
and the momentum-exchange force is differentiable with respect to q
(emb_mex_force_backward).
"""
from __future__ import annotations

import torch

from .emb import Embedding, embed, emb_cutlinks_backward, emb_mex_force, emb_mex_force_backward


class CutLinkQ(torch.autograd.Function):
    """q of every cut link as a function of the vertex positions (world units)."""

    @staticmethod
    def forward(ctx, verts: torch.Tensor, E: Embedding):
        ctx.E = E
        return E.links["q"].clone()

    @staticmethod
    def backward(ctx, gq: torch.Tensor):
        E = ctx.E
        L = E.links
        gv = emb_cutlinks_backward(E.mesh, E.forest, L["cell"], L["dir"], L["q"], L["tri"], gq.contiguous())
        return gv, None


class MexForce(torch.autograd.Function):
    """Momentum-exchange force (3 floats) on the body from populations `pop` [Q, cells]."""

    @staticmethod
    def forward(ctx, q: torch.Tensor, E: Embedding, pop: torch.Tensor):
        L = E.links
        qd = q.detach().contiguous()
        ctx.E, ctx.pop, ctx.q = E, pop, qd
        return emb_mex_force(E.forest, E.lattice, L["cell"], L["dir"], qd, pop)

    @staticmethod
    def backward(ctx, gF: torch.Tensor):
        E = ctx.E
        L = E.links
        gq = emb_mex_force_backward(E.forest, E.lattice, L["cell"], L["dir"], ctx.q, ctx.pop, gF.contiguous())
        return gq, None, None


def embed_q(verts: torch.Tensor, tris: torch.Tensor, R: int, levels: int, band: int = 2, lattice: int = 19,
            **kw):
    """Runs the embedding and returns (Embedding, q) with q attached to `verts` for autograd."""
    E = embed(verts.detach(), tris, R, levels, band, lattice, **kw)
    return E, CutLinkQ.apply(verts, E)


def mex_force(q: torch.Tensor, E: Embedding, pop: torch.Tensor) -> torch.Tensor:
    return MexForce.apply(q, E, pop)
