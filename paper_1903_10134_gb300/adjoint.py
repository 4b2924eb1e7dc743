"""Differentiable mDPD: gradients through velocity-Verlet windows and through
one evaluation, for single systems and batches of replicas.

`window(system, params, x0, v0, A, B, gamma, nsteps, step0)` advances the
system `nsteps` steps of Algorithm 1 from (x0, v0) with the pair tables A, B,
gamma and returns (x_K, v_K) -- or, with `observables=True`, also the final
evaluation's local densities rho_K (Sec. 2.1) and conservative virial W_K
(six components per replica, the pressure tensor's interaction part of Sec.
4.1) -- as a differentiable function of (x0, v0, A, B, gamma).  The forward
records the window's checkpoints in the library (`mdpd_window_forward`); the
backward runs the window's chain rule in reverse with one force VJP per step,
the random stream of every step held fixed (`mdpd_window_vjp_dev`).  Every
step of the method, forward and backward, runs in the library's kernels; this
module only moves tensors between torch.autograd and the C ABI.

For a single system A, B, gamma are (8, 8) tables and W_K is (6,); for a
batch (a `mdpd.Batch`) they are (nrep, 8, 8) and (nrep, 6), and `params` is
the list of the replicas' parameters (only their tables are replaced).
Reflection off walls or non-periodic faces is not differentiable; such
systems are refused.  After the backward the system is back at the start of
the window.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mdpd as M


def _is_batch(system) -> bool:
    return isinstance(system, M.Batch)


def _set_tables(system, params, A, B, G):
    """Write the tables A, B, gamma into the handle's parameters."""
    if _is_batch(system):
        ps = []
        for r, p in enumerate(params):
            q = p.copy()
            q.A = A[r].detach().double().cpu().numpy().copy()
            q.B = B[r].detach().double().cpu().numpy().copy()
            q.gamma = G[r].detach().double().cpu().numpy().copy()
            ps.append(q)
        M.mdpd_batch_set_params(system.h, ps)
    else:
        q = params.copy()
        q.A = A.detach().double().cpu().numpy().copy()
        q.B = B.detach().double().cpu().numpy().copy()
        q.gamma = G.detach().double().cpu().numpy().copy()
        M.mdpd_set_params(system.h, q)


def _virial(system, device):
    """Conservative virial of the last evaluation, (6,) or (nrep, 6)."""
    if _is_batch(system):
        obs = M.mdpd_batch_observables(system.h, False, False)
        return torch.tensor(np.ascontiguousarray(obs[:, 5:11]), dtype=torch.float64, device=device)
    obs = M.mdpd_observables(system.h)
    return torch.tensor(np.ascontiguousarray(obs[5:11]), dtype=torch.float64, device=device)


def _opt(t):
    """A contiguous cotangent, or None (zero) when autograd passes none."""
    return t.contiguous() if t is not None else None


class _Window(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, A, B, G, system, params, nsteps, step0):
        h = system.h
        _set_tables(system, params, A, B, G)
        M.mdpd_set_step(h, step0)
        M.mdpd_set_state_dev(h, x0.detach().contiguous(), v0.detach().contiguous())
        M.mdpd_window_forward(h, nsteps)
        x = torch.empty_like(x0)
        v = torch.empty_like(v0)
        rho = torch.empty(x0.shape[0], dtype=torch.float64, device=x0.device)
        M.mdpd_get_state_dev(h, x, v, None, rho)
        W = _virial(system, x0.device)
        ctx.system = system
        ctx.tshape = tuple(A.shape)
        return x, v, rho, W

    @staticmethod
    def backward(ctx, xbar, vbar, rhobar, wbar):
        system = ctx.system
        h = system.h
        like = torch.empty((system.n, 3), dtype=torch.float64, device=(
            xbar if xbar is not None else vbar if vbar is not None else rhobar
            if rhobar is not None else wbar).device)
        x0b = torch.empty_like(like)
        v0b = torch.empty_like(like)
        nrep = system.nrep if _is_batch(system) else 1
        tb = torch.empty((nrep, 3, 8, 8), dtype=torch.float64, device=like.device)
        M.mdpd_window_vjp_dev(h, _opt(xbar), _opt(vbar), _opt(wbar), _opt(rhobar), x0b, v0b, tb)
        if _is_batch(system):
            gA, gB, gG = tb[:, 0], tb[:, 1], tb[:, 2]
        else:
            gA, gB, gG = tb[0, 0], tb[0, 1], tb[0, 2]
        return x0b, v0b, gA, gB, gG, None, None, None, None


def window(system, params, x0, v0, A, B, gamma, nsteps: int, step0: int = 0,
           observables: bool = False):
    """Differentiable (x_K, v_K) after nsteps velocity-Verlet steps, and with
    observables=True also (rho_K, W_K) of the last evaluation (see module)."""
    x, v, rho, W = _Window.apply(x0, v0, A, B, gamma, system, params, int(nsteps), int(step0))
    return (x, v, rho, W) if observables else (x, v)


def eval_vjp(system, abar=None, cvir=None, rhobar=None):
    """(xbar, ubar, theta_bar) of one evaluation at the system's current
    state (mdpd_eval_vjp_dev): L = sum abar . a + sum cvir . W + sum rhobar rho."""
    ref = next(t for t in (abar, cvir, rhobar) if t is not None)
    n = system.n
    nrep = system.nrep if _is_batch(system) else 1
    xb = torch.empty((n, 3), dtype=torch.float64, device=ref.device)
    ub = torch.empty_like(xb)
    tb = torch.empty((nrep, 3, 8, 8), dtype=torch.float64, device=ref.device)
    M.mdpd_eval_vjp_dev(system.h, None if abar is None else abar.contiguous(),
                        None if cvir is None else cvir.contiguous(),
                        None if rhobar is None else rhobar.contiguous(), xb, ub, tb)
    return xb, ub, (tb if _is_batch(system) else tb[0])


def force_vjp(system, abar: torch.Tensor):
    """(xbar, ubar, theta_bar) of one force evaluation at the system's current
    positions, velocities and step index."""
    return eval_vjp(system, abar=abar)


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
