"""Gradients of a loss on the final displacement with respect to a per-node shear modulus and the
body force, as a torch.autograd.Function over a simulation.

The forward pass runs the steps, saving the state every `every` steps.  The backward pass seeds
the reverse sweep with dL/du(t_N), then walks the saved states from the last to the first: it
restores one, recomputes the steps up to the next saved state, each recording the F it recovers
(lbm_step_moments: D*D values per node), and reverses those steps in the opposite order
(lbm_adjoint_step).  Memory: ceil(N/every) saved states plus `every` recorded F fields, the
latter kept on the simulation for later sweeps.  All arithmetic runs in the library's kernels;
this module orders the calls.  The initial populations are held fixed: from rest with F = I they do
not depend on mu or b and the gradients are complete.
"""
from __future__ import annotations

import torch

from . import lbm


def _ring(sim: "lbm.Simulation", every: int):
    ring = getattr(sim, "_adj_ring", None)
    if ring is None or len(ring) < every:
        nb = sim.moments_bytes()
        ring = [torch.empty(nb, dtype=torch.uint8, device=sim.device) for _ in range(every)]
        sim._adj_ring = ring
    return ring


class DisplacementRun(torch.autograd.Function):
    """u(t_N) of `sim` as a function of (mu, b); `sim` must be created with adjoint=True on a body
    with velocity-Dirichlet cut links only."""

    @staticmethod
    def forward(ctx, mu: torch.Tensor, b: torch.Tensor, sim: "lbm.Simulation", nsteps: int, every: int):
        sim.set_mu_field(mu.detach())
        sim.set_body_force([float(x) for x in b.detach().cpu()])
        sim.set_initial()
        saved = []
        done = 0
        while done < nsteps:
            saved.append(sim.save_state())
            k = min(every, nsteps - done)
            sim.step(k)
            done += k
        final = sim.save_state()
        _, _, u = sim.fields()
        ctx.sim, ctx.saved, ctx.final, ctx.nsteps, ctx.every = sim, saved, final, nsteps, every
        ctx.b_shape = b.shape
        return u.clone()

    @staticmethod
    def backward(ctx, grad_u: torch.Tensor):
        sim, saved, nsteps, every = ctx.sim, ctx.saved, ctx.nsteps, ctx.every
        ring = _ring(sim, every)
        sim.load_state(ctx.final)
        sim.adjoint_begin(grad_u)
        for s in reversed(range(len(saved))):
            n0 = s * every
            n1 = min(n0 + every, nsteps)
            sim.load_state(saved[s])
            for i in range(n1 - n0):
                sim.step_moments(ring[i])
            for i in reversed(range(n1 - n0)):
                sim.adjoint_step(ring[i])
        gm, gb = sim.adjoint_gradients()
        gbt = torch.as_tensor(gb[: ctx.b_shape.numel()], dtype=torch.float64).reshape(ctx.b_shape)
        return gm, gbt, None, None, None


def displacement(mu: torch.Tensor, b: torch.Tensor, sim: "lbm.Simulation", nsteps: int, every: int = 100):
    """u (D, *box) after nsteps steps, differentiable with respect to mu (box-shaped) and b (D)."""
    return DisplacementRun.apply(mu, b, sim, nsteps, every)
