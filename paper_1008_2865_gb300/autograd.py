"""torch.autograd.Function around the library's adjoint (lb_adjoint).

    J = LBObjective.apply(rho_init, G1, G2, rho_target, steps)
    J.backward()      # rho_init.grad, G1.grad, G2.grad

J = E_s(T) + E_m(T) + sum_x (rho(x, T) - rho*(x))^2 after `steps` steps of the
two-belt Shan–Chen lattice from f = w rho_init (FP32 state, FP64 gradient
accumulation; see include/lb.h, lb_adjoint). When any input needs a gradient,
the forward pass runs the library's checkpointed reverse sweep at once and
keeps the gradients for backward; otherwise it steps forward and evaluates J
with lb_objective, the adjoint's own terminal kernel, so both paths give the
same J bit for bit. All arithmetic runs in the library's CUDA kernels; torch
only moves tensors.
"""
from __future__ import annotations

import torch

from . import Lattice


class LBObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho_init, G1, G2, rho_target, steps, omega=1.0, rho0=1.0,
                checkpoint_every=0, device=0):
        rho = rho_init.detach().to(torch.float64).contiguous()
        tgt = rho_target.detach().to(torch.float64).contiguous()
        need = any(ctx.needs_input_grad[:3])
        with Lattice(rho, omega=omega, G1=float(G1), G2=float(G2), rho0=rho0, prec="fp32",
                     trace_every=0, device=device) as lat:
            if need:
                grad = torch.empty_like(rho)
                J, _, gG = lat.adjoint(int(steps), tgt, checkpoint_every, grad_rho=grad)
                ctx.save_for_backward(grad, torch.tensor(gG, dtype=torch.float64))
            else:
                # J only: steps, then the adjoint's terminal sums on the device
                lat.step(int(steps))
                J = lat.objective(tgt)
        return torch.tensor(J, dtype=torch.float64, device=rho_init.device)

    @staticmethod
    def backward(ctx, gJ):
        grad, gG = ctx.saved_tensors
        g = gJ.to(grad.device)
        d_rho = (g * grad).to(grad.dtype) if ctx.needs_input_grad[0] else None
        d_g1 = (gJ.cpu() * gG[0]) if ctx.needs_input_grad[1] else None
        d_g2 = (gJ.cpu() * gG[1]) if ctx.needs_input_grad[2] else None
        return d_rho, d_g1, d_g2, None, None, None, None, None, None
