"""torch.autograd.Function over the library's energy and its adjoint.

Forward: E(U; R, Z) of Eq. (energy) for an orbital block U (not
orthonormalised) and Gaussian-well atoms (R, Z).  Backward: the adjoint
kernels give dE/dU = 2 f dV H(rho_U) U (E_{u_i} = H u_i, Sec. 2.1) and the
atom gradients dE/dR, dE/dZ; the Hartree and exchange potentials are rebuilt
from rho(U) inside the backward call, nothing per-orbital is saved.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pou


class KohnShamEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, R, Z, solver, width):
        solver.set_atoms(R.detach().cpu().numpy(), Z.detach().cpu().numpy(), width)
        terms = solver.evaluate(U.detach().contiguous())
        ctx.save_for_backward(U, R, Z)
        ctx.solver = solver
        ctx.width = width
        return torch.tensor(terms["total"], dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gE):
        U, R, Z = ctx.saved_tensors
        solver = ctx.solver
        solver.set_atoms(R.detach().cpu().numpy(), Z.detach().cpu().numpy(), ctx.width)
        g = float(gE.detach().cpu())
        need_u = ctx.needs_input_grad[0]
        need_atoms = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        dU = torch.empty_like(U) if need_u else None
        Uc = U.detach().contiguous()
        _, dR, dZ = solver.backward(Uc, g, dU, atoms=need_atoms)
        gR = torch.from_numpy(dR).to(R.device, R.dtype) if ctx.needs_input_grad[1] else None
        gZ = torch.from_numpy(dZ).to(Z.device, Z.dtype) if ctx.needs_input_grad[2] else None
        return dU, gR, gZ, None, None


def kohn_sham_energy(U, R, Z, solver, width=0.8):
    """Differentiable E(U, R, Z) computed by the GPU library."""
    return KohnShamEnergy.apply(U, R, Z, solver, width)
