"""torch.autograd interface of the nonbonded forces.

``NonbondedForces`` runs nb_forces in its forward pass and the hand-written
adjoint nb_backward in its backward pass, so that a loss of the forces (for
example force matching) can be differentiated with respect to positions,
charges and the LJ matrix. The per-type -> pair-matrix combination rule
(C_ab = sqrt(c_a c_b)) is plain torch (``lj_matrix``), so gradients flow on
to per-type parameters. Energies are returned but are not differentiable.
"""
from __future__ import annotations

import torch

from . import nb


class NonbondedForces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, q, ljparams, pairlist, type_, rc, beta):
        lj32 = ljparams.detach().to(torch.float32).contiguous()
        F = torch.empty((pairlist.n_atoms, 3), dtype=torch.float32, device=coords.device)
        E = torch.empty(2, dtype=torch.float64, device=coords.device)
        pairlist.forces(coords.detach().contiguous(), q.detach().to(torch.float32).contiguous(), type_, lj32, rc,
                        beta, F, E)
        ctx.save_for_backward(coords, q, lj32, type_)
        ctx.pairlist = pairlist
        ctx.rc = float(rc)
        ctx.beta = float(beta)
        ctx.lj_dtype = ljparams.dtype
        ctx.q_dtype = q.dtype
        ctx.mark_non_differentiable(E)
        return F, E

    @staticmethod
    def backward(ctx, gF, gE):
        coords, q, lj32, type_ = ctx.saved_tensors
        gx, gq, glj = ctx.pairlist.backward(coords.detach().contiguous(), q.detach().to(torch.float32).contiguous(),
                                            type_, lj32, ctx.rc, ctx.beta, gF.to(torch.float32).contiguous())
        return (gx if ctx.needs_input_grad[0] else None,
                gq.to(ctx.q_dtype) if ctx.needs_input_grad[1] else None,
                glj.to(ctx.lj_dtype) if ctx.needs_input_grad[2] else None,
                None, None, None, None)


def lj_matrix(c6: torch.Tensor, c12: torch.Tensor) -> torch.Tensor:
    """Per-type (c6, c12) -> [ntype, ntype, 2] pair matrix, C_ab = sqrt(c_a c_b)."""
    return torch.stack([torch.sqrt(torch.outer(c6, c6)), torch.sqrt(torch.outer(c12, c12))], dim=-1)


def nonbonded_forces(coords, q, ljparams, pairlist: nb.Pairlist, type_, rc: float, beta: float):
    """Forces [N, 3] (differentiable) and energies [2] (E_LJ, E_C) of the current pair list."""
    return NonbondedForces.apply(coords, q, ljparams, pairlist, type_, rc, beta)


def force_matching_loss(forces: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """(1/3N) sum_i |F_i - T_i|^2."""
    return ((forces.to(torch.float64) - target.to(torch.float64)) ** 2).mean()
