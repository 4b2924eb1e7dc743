"""Gradients through short velocity-Verlet windows of the mDPD dynamics.

`window(system, params, x0, v0, A, B, gamma, nsteps, step0)` advances the
library's system `nsteps` steps from (x0, v0) with the pair tables A, B, gamma
and returns (x_K, v_K) as a differentiable function of (x0, v0, A, B, gamma):
`torch.autograd.Function` whose backward undoes the steps in reverse with the
library's force vector-Jacobian product (`mdpd_force_vjp_dev`, hand-written
CUDA kernels), the random stream of every step held fixed.  The forward keeps
the positions and half-step velocities of every step (step checkpoints).

The chain rule per step, with (xb, vb, ab) the adjoints of
(x_{k+1}, v_{k+1}, a_{k+1}) and h = dt/2:
    v_{k+1} = v'_k + h a_{k+1}   ->  vhb = vb,  ab += h vb
    a_{k+1} = F(x_{k+1}, v'_k)   ->  xb += F_x^T ab, vhb += F_u^T ab, theta_bar += F_theta^T ab
    x_{k+1} = x_k + dt v'_k      ->  vhb += dt xb
    v'_k = v_k + h a_k           ->  vb = vhb, ab = h vhb
and finally a_0 = F(x_0, v_0).  Frozen particles neither kick nor drift.
Reflection off walls is not differentiable; systems with a wall mask are
refused.  The system's state is overwritten by the backward pass.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mdpd as M


def _mobile_mask(system, params, device):
    _, _, typ, _ = system.state()
    mob = np.array([((params.frozen_mask >> int(t)) & 1) == 0 for t in typ], dtype=np.float64)
    return torch.tensor(mob, device=device).unsqueeze(1)


def force_vjp(system, abar: torch.Tensor):
    """(xbar, ubar, theta_bar) of one force evaluation at the system's current
    positions, velocities and step index."""
    xb = torch.zeros_like(abar)
    ub = torch.zeros_like(abar)
    tb = torch.zeros((3, 8, 8), dtype=torch.float64, device=abar.device)
    M.mdpd_force_vjp_dev(system.h, abar.contiguous(), xb, ub, tb)
    return xb, ub, tb


def _vjp_at(system, x, u, step, abar):
    M.mdpd_set_step(system.h, step)
    M.mdpd_set_state_dev(system.h, x.contiguous(), u.contiguous())
    return force_vjp(system, abar)


class _Window(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, A, B, G, system, params, nsteps, step0):
        if getattr(system, "has_walls", False):
            raise ValueError("reflection off walls is not differentiable")
        p = params.copy()
        p.A = A.detach().double().cpu().numpy().copy()
        p.B = B.detach().double().cpu().numpy().copy()
        p.gamma = G.detach().double().cpu().numpy().copy()
        h = system.h
        M.mdpd_set_params(h, p)
        M.mdpd_set_step(h, step0)
        M.mdpd_set_state_dev(h, x0.detach().contiguous(), v0.detach().contiguous())
        mob = _mobile_mask(system, p, x0.device)
        hdt = 0.5 * p.dt
        a = torch.empty_like(x0)
        M.mdpd_get_accel_dev(h, a)
        v = v0.detach()
        xs, vhs = [], []
        x = x0.detach()
        for _ in range(nsteps):
            vhs.append(v + hdt * a * mob)
            M.mdpd_step(h, 1)
            x = torch.empty_like(x0)
            v = torch.empty_like(v0)
            M.mdpd_get_state_dev(h, x, v)
            M.mdpd_get_accel_dev(h, a)
            xs.append(x)
        ctx.system, ctx.params, ctx.step0, ctx.mob = system, p, step0, mob
        ctx.x0, ctx.v0, ctx.xs, ctx.vhs = x0.detach(), v0.detach(), xs, vhs
        return x.clone(), v.clone()

    @staticmethod
    def backward(ctx, xbar, vbar):
        system, p, s0, mob = ctx.system, ctx.params, ctx.step0, ctx.mob
        h, dt = 0.5 * p.dt, p.dt
        xb = xbar.double().clone() if xbar is not None else torch.zeros_like(ctx.x0)
        vb = vbar.double().clone() if vbar is not None else torch.zeros_like(ctx.v0)
        ab = torch.zeros_like(xb)
        tb = torch.zeros((3, 8, 8), dtype=torch.float64, device=xb.device)
        for k in range(len(ctx.xs) - 1, -1, -1):
            vhb = vb.clone()
            ab = ab + h * vb * mob
            gx, gu, gt = _vjp_at(system, ctx.xs[k], ctx.vhs[k], s0 + k + 1, ab)
            xb = xb + gx
            vhb = vhb + gu
            tb = tb + gt
            vhb = vhb + dt * xb * mob
            vb = vhb
            ab = h * vhb * mob
        gx, gu, gt = _vjp_at(system, ctx.x0, ctx.v0, s0, ab)
        xb, vb, tb = xb + gx, vb + gu, tb + gt
        return xb, vb, tb[0], tb[1], tb[2], None, None, None, None


class _Density(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, system):
        zero = torch.zeros_like(x)
        M.mdpd_set_state_dev(system.h, x.detach().contiguous(), zero)
        rho = torch.empty(x.shape[0], dtype=torch.float64, device=x.device)
        M.mdpd_forces_dev(system.h, None, rho)
        ctx.system = system
        ctx.save_for_backward(x.detach())
        return rho

    @staticmethod
    def backward(ctx, rbar):
        (x,) = ctx.saved_tensors
        M.mdpd_set_state_dev(ctx.system.h, x.contiguous(), torch.zeros_like(x))
        xb = torch.empty_like(x)
        M.mdpd_density_vjp_dev(ctx.system.h, rbar.double().contiguous(), xb)
        return xb, None


def density(system, x):
    """Differentiable local densities rho_i (Sec. 2.1) of the system's particles
    at positions x (N x 3, device): forward through the density pass, backward
    through its vector-Jacobian product (mdpd_density_vjp_dev).  The system's
    state is overwritten (positions x, velocities zero)."""
    return _Density.apply(x, system)


def window(system, params, x0, v0, A, B, gamma, nsteps: int, step0: int = 0):
    """Differentiable (x_K, v_K) after nsteps velocity-Verlet steps (see module)."""
    return _Window.apply(x0, v0, A, B, gamma, system, params, int(nsteps), int(step0))
