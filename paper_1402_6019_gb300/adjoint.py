"""Gradients of a run through the discrete adjoint of the step (library kernels, FP64).

A run is f_0 = W_l rho_init (the state lbm_set_fields makes with u = 0), then
f_{n+1} = S(f_n; theta) for `steps` steps, scored by the velocity / density profile objective
of lbm_adjoint_objective (targets of the kind Sec. IV measures: the x-averaged stream-flow
velocity and the density of species A across the channel).  theta holds the NPARAM model
parameters in the order of the adjoint entry points:
G1 A, G1 B, G2 A, G2 B, G_AB, tau A, tau B, body_force.

The backward sweep needs every state f_n in reverse order.  Storing them all takes
steps x 9 ns nx nz doubles, so the forward keeps a copy every `checkpoint` steps and the
backward recomputes one segment at a time from its copy (lbm_set_populations, then single
steps): device memory for ceil(steps / checkpoint) + checkpoint states, and one extra forward
run.  Every step, objective and adjoint step runs in the library; this module only orders the
calls and holds the buffers.
"""
from __future__ import annotations

import torch

from . import lbm as L

NPARAM = 8
_KEYS = [("G1", 0), ("G1", 1), ("G2", 0), ("G2", 1), ("G_AB", None), ("tau", 0), ("tau", 1), ("body_force", None)]


def theta_of(p: L.lbm_params) -> list:
    """The NPARAM parameters of p, in the adjoint's order."""
    return [getattr(p, k)[i] if i is not None else getattr(p, k) for k, i in _KEYS]


def set_theta(lat: L.Lattice, theta) -> None:
    """Write theta into the lattice's parameters (the other parameters are kept)."""
    p = lat.params
    for (k, i), v in zip(_KEYS, [float(t) for t in theta]):
        if i is None:
            setattr(p, k, v)
        else:
            getattr(p, k)[i] = v
    L.lbm_set_params(lat.h, p)


def _state(lat):
    f = torch.empty((lat.ns, 9, lat.nz, lat.nx), dtype=torch.float64, device=f"cuda:{lat.desc.device}")
    L.lbm_get_fields(lat.h, f=f)
    return f


def forward_run(lat: L.Lattice, rho_init: torch.Tensor, steps: int, checkpoint: int):
    """Run from the state at rest with densities rho_init; returns (final state, checkpoints)."""
    if checkpoint < 1:
        raise ValueError("checkpoint must be >= 1")
    lat.set_fields(rho_init.contiguous())
    ckpts = []
    for k in range(0, steps, checkpoint):
        ckpts.append(_state(lat))
        lat.step(min(checkpoint, steps - k))
    return _state(lat), ckpts


def objective(lat: L.Lattice, f: torch.Tensor, target_u: torch.Tensor, target_rho: torch.Tensor, grad=True):
    """(J as a 0-d device tensor, dJ/df or None)."""
    J = torch.zeros((), dtype=torch.float64, device=f.device)
    g = torch.empty_like(f) if grad else None
    L.lbm_adjoint_objective(lat.h, f, target_u.contiguous(), target_rho.contiguous(), J, g)
    return J, g


def backward_run(lat: L.Lattice, ckpts, steps: int, checkpoint: int, lam: torch.Tensor):
    """lam = dJ/df_steps in; returns (dJ/drho_init, dJ/dtheta) after sweeping every step back."""
    grad = torch.zeros(NPARAM, dtype=torch.float64, device=lam.device)
    seg = [torch.empty_like(lam) for _ in range(min(checkpoint, steps))]
    nxt = torch.empty_like(lam)
    for k in reversed(range(len(ckpts))):
        n = min(checkpoint, steps - k * checkpoint)
        lat.set_populations(ckpts[k])
        for j in range(n):  # recompute the segment's states
            L.lbm_get_fields(lat.h, f=seg[j])
            lat.step(1)
        for j in reversed(range(n)):
            L.lbm_adjoint_step(lat.h, seg[j], lam, nxt, grad)
            lam, nxt = nxt, lam
    g_rho = torch.empty((lat.ns, lat.nz, lat.nx), dtype=torch.float64, device=lam.device)
    L.lbm_adjoint_initial(lat.h, lam, g_rho)
    lat.synchronize()
    return g_rho, grad


def rollout_gradient(lat: L.Lattice, rho_init: torch.Tensor, steps: int, target_u: torch.Tensor,
                     target_rho: torch.Tensor, checkpoint: int = 25):
    """(J, dJ/drho_init [ns, nz, nx], dJ/dtheta [NPARAM]) of a run of `steps` steps."""
    fN, ckpts = forward_run(lat, rho_init, steps, checkpoint)
    J, lam = objective(lat, fN, target_u, target_rho)
    g_rho, grad = backward_run(lat, ckpts, steps, checkpoint, lam)
    return float(J), g_rho, grad


class ProfileLoss(torch.autograd.Function):
    """J(rho_init, theta) of a run as a differentiable torch function.

    ProfileLoss.apply(lat, rho_init, theta, target_u, target_rho, steps, checkpoint): rho_init a
    CUDA float64 tensor [ns, nz, nx], theta a float64 tensor of NPARAM parameters (written into
    the lattice's parameters).  The backward pass recomputes the run from its checkpoints and
    sweeps the adjoint, returning the gradients for rho_init and theta."""

    @staticmethod
    def forward(ctx, lat, rho_init, theta, target_u, target_rho, steps, checkpoint):
        set_theta(lat, theta.detach().cpu().tolist())
        fN, ckpts = forward_run(lat, rho_init.detach(), steps, checkpoint)
        J, lam = objective(lat, fN, target_u, target_rho)
        ctx.lat, ctx.steps, ctx.checkpoint = lat, steps, checkpoint
        ctx.ckpts, ctx.lam = ckpts, lam
        ctx.theta_device = theta.device
        return J

    @staticmethod
    def backward(ctx, gJ):
        g_rho, grad = backward_run(ctx.lat, ctx.ckpts, ctx.steps, ctx.checkpoint, ctx.lam)
        ctx.ckpts = ctx.lam = None
        return None, gJ * g_rho, (gJ * grad).to(ctx.theta_device), None, None, None, None
