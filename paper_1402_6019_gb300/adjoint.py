"""Gradients of a run through the discrete adjoint of the step (library kernels).

A run is f_0 = W_l rho_init (the state lbm_set_fields makes with u = 0), then
f_{n+1} = S(f_n; theta) for `steps` steps, scored by the velocity / density profile objective
of lbm_adjoint_objective (targets of the kind Sec. IV measures: the x-averaged stream-flow
velocity and the density of species A across the lattice).  theta holds the NPARAM model
parameters in the order of the adjoint entry points:
G1 A, G1 B, G2 A, G2 B, G_AB, tau A, tau B, body_force.

The backward sweep needs every state f_n in reverse order.  Storing them all takes
steps x 9 ns nx nz values, so the forward keeps an exact snapshot every `checkpoint` steps and
the backward recomputes one segment at a time from its snapshot (lbm_restore_own, then
lbm_record_states), sweeping it back with lbm_adjoint_steps: device memory for
ceil(steps / checkpoint) snapshots and `checkpoint` recorded states, and one extra forward run.

The adjoint runs in the lattice's precision unless told otherwise: an FP32 lattice records FP32
states and sweeps an FP32 adjoint; the parameter derivatives are accumulated in FP64 either way.
Every step, objective and adjoint step runs in the library; this module orders the calls and
holds the buffers.
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


def _dtype(lat, dtype):
    if dtype is not None:
        return dtype
    return torch.float32 if lat.desc.precision == L.LBM_FP32 else torch.float64


def _device(lat):
    return torch.device("cuda", lat.desc.device)


def _handoff(device):
    """Wait for torch's work on its current stream: the library runs on the lattice's own
    stream, so tensors torch just wrote must be complete before the library reads them."""
    torch.cuda.current_stream(device).synchronize()


class Run:
    """The forward run of a gradient: snapshots every `checkpoint` steps and the final state."""

    def __init__(self, lat: L.Lattice, rho_init: torch.Tensor, steps: int, checkpoint: int, dtype=None):
        if checkpoint < 1 or steps < 0:
            raise ValueError("checkpoint must be >= 1 and steps >= 0")
        self.lat, self.steps, self.checkpoint = lat, steps, checkpoint
        self.dtype = _dtype(lat, dtype)
        rho_init = rho_init.detach().contiguous()
        _handoff(_device(lat))
        lat.set_fields(rho_init)
        nb = L.lbm_snapshot_bytes(lat.h)
        self.snaps = []
        for k in range(0, steps, checkpoint):
            s = torch.empty(nb, dtype=torch.uint8, device=_device(lat))
            L.lbm_snapshot(lat.h, s)
            self.snaps.append(s)
            lat.step(min(checkpoint, steps - k))
        self.final = torch.empty((lat.ns, 9, lat.nz, lat.nx), dtype=self.dtype, device=_device(lat))
        L.lbm_export_state(lat.h, self.final)

    def objective(self, target_u, target_rho, grad=True):
        """(J as a 0-d FP64 device tensor, dJ/df_steps or None); synchronises."""
        J = torch.empty((), dtype=torch.float64, device=self.final.device)
        g = torch.empty_like(self.final) if grad else None
        target_u, target_rho = target_u.contiguous(), target_rho.contiguous()
        _handoff(self.final.device)
        L.lbm_adjoint_objective(self.lat.h, self.final, target_u, target_rho, J, g)
        self.lat.synchronize()
        return J, g

    def backward(self, lam: torch.Tensor):
        """lam = dJ/df_steps; returns (dJ/drho_init [ns, nz, nx], dJ/dtheta [NPARAM]), FP64."""
        lat = self.lat
        lam = lam.to(self.dtype).contiguous().clone()
        grad = torch.zeros(NPARAM, dtype=torch.float64, device=lam.device)
        seg = torch.empty((min(self.checkpoint, max(self.steps, 1)),) + tuple(lam.shape), dtype=self.dtype,
                          device=lam.device)
        _handoff(lam.device)
        for k in reversed(range(len(self.snaps))):
            n = min(self.checkpoint, self.steps - k * self.checkpoint)
            L.lbm_restore_own(lat.h, self.snaps[k])
            L.lbm_record_states(lat.h, n, seg)
            L.lbm_adjoint_steps(lat.h, n, seg, lam, grad)
        g_rho = torch.empty((lat.ns, lat.nz, lat.nx), dtype=torch.float64, device=lam.device)
        L.lbm_adjoint_initial(lat.h, lam, g_rho)
        lat.synchronize()
        return g_rho, grad


def rollout_gradient(lat: L.Lattice, rho_init: torch.Tensor, steps: int, target_u: torch.Tensor,
                     target_rho: torch.Tensor, checkpoint: int = 25, dtype=None):
    """(J, dJ/drho_init [ns, nz, nx], dJ/dtheta [NPARAM]) of a run of `steps` steps."""
    run = Run(lat, rho_init, steps, checkpoint, dtype)
    J, lam = run.objective(target_u, target_rho)
    g_rho, grad = run.backward(lam)
    return float(J), g_rho, grad


def objective_value(lat: L.Lattice, rho_init: torch.Tensor, steps: int, target_u: torch.Tensor,
                    target_rho: torch.Tensor, dtype=None) -> float:
    """J of a run, without keeping snapshots or forming a gradient."""
    run = Run(lat, rho_init, steps, max(steps, 1), dtype)
    run.snaps = []
    return float(run.objective(target_u, target_rho, grad=False)[0])


class ProfileLoss(torch.autograd.Function):
    """J(rho_init, theta) of a run as a differentiable torch function.

    ProfileLoss.apply(lat, rho_init, theta, target_u, target_rho, steps, checkpoint): rho_init a
    CUDA float64 tensor [ns, nz, nx], theta a float64 tensor of NPARAM parameters (written into
    the lattice's parameters).  The backward pass recomputes the run from its snapshots and
    sweeps the adjoint, returning the gradients for rho_init and theta."""

    @staticmethod
    def forward(ctx, lat, rho_init, theta, target_u, target_rho, steps, checkpoint):
        set_theta(lat, theta.detach().cpu().tolist())
        run = Run(lat, rho_init, steps, checkpoint)
        J, lam = run.objective(target_u, target_rho)
        ctx.run, ctx.lam, ctx.theta_device = run, lam, theta.device
        return J

    @staticmethod
    def backward(ctx, gJ):
        g_rho, grad = ctx.run.backward(ctx.lam)
        ctx.run = ctx.lam = None
        return None, gJ * g_rho, (gJ * grad).to(ctx.theta_device), None, None, None, None
