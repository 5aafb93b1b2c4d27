"""Differentiable subdivision: a torch.autograd.Function around libalsub.

Vertex refinement is linear in the control positions (P_L = R P_0, Sec. 3.6 Eq. singleSpMV), so
the gradient of any loss of P_L is g_0 = R^T g_L. Forward runs the fused eval kernels
(alsub_refine_vertices); backward applies the transposed per-level operators
g_l = R_l^T g_{l+1} (alsub_apply_operator_transpose), which depend on the topology only: no
intermediate positions are kept for the backward pass. A closed Catmull-Clark mesh applies them
matrix-free, gathered per coarse vertex (ALSUB_OP_MATRIX_FREE); other meshes through their stored
transposes (ALSUB_OP_TRANSPOSE). Feature-adaptive refinement (Sec. 3.4) is differentiated the same
way through its composed operator R = R^(n) X^(n) ... R^(1) X^(1) and the stored R^T.
"""
from __future__ import annotations

import torch

from . import alsub


class Refine(torch.autograd.Function):
    """P_L = refine(P_0) on a fixed topology; d/dP_0 = R^T."""

    @staticmethod
    def forward(ctx, P0: torch.Tensor, topo: alsub.Topology, op: alsub.Operator):
        ctx.op = op
        return topo.refine_vertices(P0.detach().contiguous())

    @staticmethod
    def backward(ctx, gL: torch.Tensor):
        return ctx.op.apply_transpose(gL.contiguous()), None, None


class Subdivider:
    """A topology plus its transposed per-level operators, ready for forward and backward."""

    def __init__(self, mesh: dict, levels: int | None = None, scheme: str | None = None):
        self.mesh = alsub.Mesh.from_dict(mesh, scheme)
        self.topo = alsub.Topology(self.mesh, levels if levels is not None else mesh["levels"])
        gather = self.mesh.scheme == "cc" and self.mesh.boundary_edges == 0
        self.op = alsub.Operator(self.topo, chain=False, matrix_free=True, transpose=not gather)

    def __call__(self, P0: torch.Tensor) -> torch.Tensor:
        return Refine.apply(P0, self.topo, self.op)


class AdaptiveRefine(torch.autograd.Function):
    """P = R P_0 for a composed feature-adaptive operator; d/dP_0 = R^T."""

    @staticmethod
    def forward(ctx, P0: torch.Tensor, op: alsub.AdaptiveOperator):
        ctx.op = op
        return op.apply(P0.detach().contiguous())

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        return ctx.op.apply_transpose(g.contiguous()), None


class AdaptiveSubdivider:
    """Rounds of (extract ``rings`` rings around the extraordinary vertices and crease ends, refine
    one level) from a control mesh, composed into one operator with its transpose; the rounds'
    topologies are released once it is built. ``stacked`` keeps every round's points."""

    def __init__(self, mesh: dict, rounds: int, rings: int = 2, scheme: str | None = None,
                 stacked: bool = False):
        M = alsub.Mesh.from_dict(mesh, scheme)
        T = alsub.Topology(M, 0)
        topos, meshes = [T], [M]
        for _ in range(rounds):
            sub = T.extract(T.levels, None, rings)
            T = alsub.Topology(sub, 1)
            topos.append(T)
            meshes.append(sub)
        self.op = alsub.AdaptiveOperator(topos, stacked=stacked, transpose=True)
        self.faces = topos[-1].faces(1)          # the last round's face table
        for t in topos:
            t.close()
        for m in meshes:
            m.close()

    def __call__(self, P0: torch.Tensor) -> torch.Tensor:
        return AdaptiveRefine.apply(P0, self.op)
