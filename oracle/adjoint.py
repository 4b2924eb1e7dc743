"""Gradient of a velocity-Verlet window by the chain rule over its steps, on
the FP64 oracle (test infrastructure only; the CUDA path has its own).

Forward window of K steps from (x_0, v_0) at step index s0, as in Algorithm 1
without communication and without walls (no reflection):
    a_0 = F(x_0, v_0; s0)
    for k = 0..K-1:
        v'_k    = v_k + (dt/2) a_k
        x_{k+1} = x_k + dt v'_k               (periodic wrap: a shift, no effect on slopes)
        a_{k+1} = F(x_{k+1}, v'_k; s0 + k + 1)
        v_{k+1} = v'_k + (dt/2) a_{k+1}
Frozen particles keep x and v.  Given xbar_K, vbar_K (the adjoints of the
final state), the steps are undone in reverse with the force VJP of each
force evaluation (random stream fixed), giving xbar_0, vbar_0 and the
gradient with respect to the symmetric parameters A, B, gamma.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def window_forward(o: "O.Oracle", nsteps: int):
    """Advance o by nsteps and return the checkpoints needed by window_vjp."""
    p = o.params
    hdt = 0.5 * p.dt
    mob = np.array([((p.frozen_mask >> int(t)) & 1) == 0 for t in o.type])[:, None]
    ck = {"s0": o.step, "x0": o.x.copy(), "v0": o.v.copy(), "x": [], "vh": [], "mob": mob}
    for _ in range(nsteps):
        vh = o.v + hdt * o.a * mob
        o.run(1)
        ck["x"].append(o.x.copy())
        ck["vh"].append(vh)
    return ck


def window_vjp(o: "O.Oracle", ck, xbar, vbar, cvir=None, rhobar=None):
    """(xbar_0, vbar_0, tbar) of the window recorded in ck.  cvir and rhobar
    (optional) are the adjoints of the conservative virial and of the local
    densities of the window's last force evaluation, a_K = F(x_K, v'_{K-1}).

    Reverse sweep, with (xb, vb, ab) the adjoints of (x_{k+1}, v_{k+1}, a_{k+1}):
      v_{k+1} = v'_k + h a_{k+1}  ->  vhb = vb,  ab += h vb
      a_{k+1} = F(x_{k+1}, v'_k)  ->  xb += F_x^T ab, vhb += F_u^T ab, tbar += F_theta^T ab
      x_{k+1} = x_k + dt v'_k     ->  vhb += dt xb   (xb carries over to x_k)
      v'_k = v_k + h a_k          ->  vb = vhb, ab = h vhb
    and finally a_0 = F(x_0, v_0).  Frozen particles neither kick nor drift
    (their x and v carry over unchanged), but their x and v still enter the
    forces on their mobile partners."""
    p = o.params
    h, dt = 0.5 * p.dt, p.dt
    mob = ck["mob"]
    xb = np.array(xbar, dtype=float)
    vb = np.array(vbar, dtype=float)
    ab = np.zeros_like(xb)
    tb = np.zeros((3, 8, 8))
    K = len(ck["x"])
    for k in range(K - 1, -1, -1):
        vhb = vb.copy()
        ab = ab + h * vb * mob
        last = k == K - 1
        gx, gu, gt = o.eval_vjp(ab, cvir if last else None, rhobar if last else None,
                                x=ck["x"][k], u=ck["vh"][k], step=ck["s0"] + k + 1)
        xb = xb + gx
        vhb = vhb + gu
        tb += gt
        vhb = vhb + dt * xb * mob
        vb = vhb
        ab = h * vhb * mob
    gx, gu, gt = o.force_vjp(ab, x=ck["x0"], u=ck["v0"], step=ck["s0"])
    return xb + gx, vb + gu, tb + gt
