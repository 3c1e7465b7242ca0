"""Differentiable Coulomb energy E(q, R) = 1/2 q . Phi(R) q over the CUDA apply.

The forward pass is one Coulomb apply (potential and field).  The backward
pass is written out by hand: dE/dq = Phi q = v (the matrix-free form
C v = u o v + dE_Coul/dv of Sec. 3.4), and dE/dR_i = -q_i E_i.  The force
includes the PME mesh-gradient path (the B-spline derivative weights of
Alg. 2, step 5).  No second apply and no graph through the kernels is needed.
That lets a machine-learned chi and eta train through the QEq energy (Sec. 4).

The neighbour list of ``system`` must be current for R (within skin / 2).
"""

from __future__ import annotations

import torch


class CoulombEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, R, sigma, system):
        v, E, F, en = system.apply(R.detach().contiguous(), q.detach().contiguous(),
                                   sigma.detach().contiguous())
        ctx.save_for_backward(v.clone(), F.clone())
        return en[0].clone()

    @staticmethod
    def backward(ctx, gE):
        v, F = ctx.saved_tensors
        gq = gE * v if ctx.needs_input_grad[0] else None
        gR = -gE * F if ctx.needs_input_grad[1] else None
        return gq, gR, None, None


def coulomb_energy(system, R, q, sigma):
    """E = 1/2 q . v, differentiable in q and R (float64 CUDA tensors)."""
    return CoulombEnergy.apply(q, R, sigma, system)
