"""Batched adjoint on the GPU: the evaluation VJP (accelerations, virial and
local densities of Sec. 2.1 / Eq. 1 and Sec. 4.1) on batches of uneven
replicas against the oracle, its determinism, 50-step velocity-Verlet windows
of a 64-replica batch against central finite differences and against the
oracle's window gradient, and a fit of (A, B) to a target density and
surface tension."""
import numpy as np
import pytest

from oracle import adjoint as OAD
from oracle import oracle as O
from paper_1903_10134_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10134_gb300 import adjoint as AD, mdpd
    mdpd.lib()
    return torch, mdpd, AD


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def _uneven_replicas(nrep, seed, ntypes=2, frozen=()):
    """Replicas of uneven box and size at number density 5 to 7 (the
    liquid's), two types with distinct tables."""
    rng = np.random.default_rng(seed)
    ws = []
    for r in range(nrep):
        L = (float(rng.uniform(3.2, 5.5)), float(rng.uniform(3.2, 5.5)), float(rng.uniform(3.2, 5.5)))
        n = int(rng.uniform(5.0, 7.0) * L[0] * L[1] * L[2])
        w = I.tiny(n, L, seed * 100 + r, ntypes=ntypes, frozen_types=frozen)
        ws.append(w)
    return ws


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 3e-4)])
def test_batch_eval_vjp_matches_oracle_per_member(env, precision, tol):
    """One launch over five uneven replicas (two types, one frozen type,
    distinct tables): every member's position, velocity and parameter
    gradients of L = abar . a + cvir . W + rhobar . rho against the oracle's
    evaluation VJP of that member alone."""
    torch, M, AD = env
    ws = _uneven_replicas(5, 3, frozen=(1,))
    b = M.Batch.from_workloads(ws, precision=precision)
    for r, w in enumerate(ws):
        assert b.n_list[r] == w.n
    rng = np.random.default_rng(4)
    abar = rng.normal(size=(b.n, 3))
    cvir = rng.normal(size=(b.nrep, 6))
    rb = rng.normal(size=b.n)
    M.mdpd_set_step(b.h, 11)
    b.set_state(np.concatenate([w.pos for w in ws]), np.concatenate([w.vel for w in ws]))
    dev = "cuda"
    xb, ub, tb = AD.eval_vjp(b, torch.tensor(abar, device=dev), torch.tensor(cvir, device=dev),
                             torch.tensor(rb, device=dev))
    xb, ub, tb = xb.cpu().numpy(), ub.cpu().numpy(), tb.cpu().numpy()
    for r, w in enumerate(ws):
        a0, a1 = b.offsets[r], b.offsets[r + 1]
        o = O.Oracle(w.params.copy(precision=0), w.pos, w.vel, w.type, w.seed, use_cells=False)
        oxb, oub, otb = o.eval_vjp(abar[a0:a1], cvir[r], rb[a0:a1], step=11)
        assert _rel(xb[a0:a1], oxb) < tol, r
        assert _rel(ub[a0:a1], oub) < tol, r
        for q in range(3):
            assert _rel(tb[r, q, :2, :2], otb[q, :2, :2]) < 10 * tol, (r, q)
    b.close()


def test_eval_vjp_is_deterministic(env):
    """The parameter gradients are reduced in a fixed order (no atomics):
    two calls give the same bits, on a single system and on a batch."""
    torch, M, AD = env
    w = I.tiny(2500, (7.0, 6.0, 6.5), 5, ntypes=2)
    s = M.System(w.params.copy(precision=1), w.pos, w.vel, w.type, w.seed)
    ab = torch.tensor(np.random.default_rng(6).normal(size=(w.n, 3)), device="cuda")
    r1 = AD.eval_vjp(s, ab)
    r2 = AD.eval_vjp(s, ab)
    for u, v in zip(r1, r2):
        assert torch.equal(u, v)
    s.close()
    ws = _uneven_replicas(6, 7)
    b = M.Batch.from_workloads(ws, precision=1)
    ab = torch.tensor(np.random.default_rng(8).normal(size=(b.n, 3)), device="cuda")
    cv = torch.tensor(np.random.default_rng(9).normal(size=(b.nrep, 6)), device="cuda")
    r1 = AD.eval_vjp(b, ab, cv)
    r2 = AD.eval_vjp(b, ab, cv)
    for u, v in zip(r1, r2):
        assert torch.equal(u, v)


def _slab_batch(nrep, seed, n_range=(600, 2000)):
    """Small liquid slabs shaped like the batched calibration's replicas."""
    return I.batch_slabs(nrep=nrep, n_range=n_range, seed=seed, precision=0)


def test_batch_window_50_steps_matches_oracle_and_finite_differences(env):
    """A 50-step window over 64 uneven slab replicas in one batch (one launch
    per kernel per step, forward and backward): the gradient of a loss on the
    final positions, velocities, virial and densities against the oracle's
    window chain rule on two members, and against central differences of the
    GPU forward along random directions of x0, v0 and per-replica A, B."""
    torch, M, AD = env
    ws = _slab_batch(64, 21)
    K = 50
    dev = "cuda"
    b = M.Batch.from_workloads(ws, precision=0)
    b.step(20)                            # leave the random start
    b.sync()
    xs, vs, _, _ = b.state()
    ps = [w.params for w in ws]
    x0 = torch.tensor(xs, device=dev, requires_grad=True)
    v0 = torch.tensor(vs, device=dev, requires_grad=True)
    A = torch.tensor(np.stack([p.A for p in ps]), device=dev, requires_grad=True)
    B = torch.tensor(np.stack([p.B for p in ps]), device=dev, requires_grad=True)
    G = torch.tensor(np.stack([p.gamma for p in ps]), device=dev, requires_grad=True)
    rng = np.random.default_rng(5)
    cx = torch.tensor(rng.normal(size=xs.shape), device=dev)
    cv = torch.tensor(rng.normal(size=xs.shape), device=dev)
    cw = torch.tensor(rng.normal(size=(b.nrep, 6)) * 1e-2, device=dev)
    cr = torch.tensor(rng.normal(size=b.n), device=dev)
    s0 = 20

    def loss_of(xk, vk, rho, W):
        return (cx * xk).sum() + (cv * vk).sum() + (cw * W).sum() + (cr * rho).sum()

    xk, vk, rho, W = AD.window(b, ps, x0, v0, A, B, G, K, step0=s0, observables=True)
    loss_of(xk, vk, rho, W).backward()
    gx0, gv0 = x0.grad.cpu().numpy(), v0.grad.cpu().numpy()
    gA, gB, gG = A.grad.cpu().numpy(), B.grad.cpu().numpy(), G.grad.cpu().numpy()

    # the oracle's chain rule on two members (the smallest and another)
    for r in (int(np.argmin(b.n_list)), 7):
        a0, a1 = b.offsets[r], b.offsets[r + 1]
        w = ws[r]
        o = O.Oracle(w.params, xs[a0:a1], vs[a0:a1], w.type, w.seed, use_cells=True, step=s0)
        ck = OAD.window_forward(o, K)
        np.testing.assert_allclose(xk.detach().cpu().numpy()[a0:a1], o.x, atol=1e-10)
        oxb, ovb, otb = OAD.window_vjp(o, ck, cx.cpu().numpy()[a0:a1], cv.cpu().numpy()[a0:a1],
                                       cvir=cw.cpu().numpy()[r], rhobar=cr.cpu().numpy()[a0:a1])
        assert _rel(gx0[a0:a1], oxb) < 1e-7, r
        assert _rel(gv0[a0:a1], ovb) < 1e-7, r
        for q, g in enumerate((gA, gB, gG)):
            assert abs(g[r, 0, 0] - otb[q, 0, 0]) <= 1e-7 * max(1.0, abs(otb[q, 0, 0])), (r, q)

    # central differences of the GPU forward
    def fwd(xx, vv, AA=None, BB=None):
        with torch.no_grad():
            out = AD.window(b, ps, xx, vv, A.detach() if AA is None else AA,
                            B.detach() if BB is None else BB, G.detach(), K, step0=s0,
                            observables=True)
            return float(loss_of(*out))

    log = []

    def fd(f, eps):
        d1 = (f(eps) - f(-eps)) / (2 * eps)
        d2 = (f(2 * eps) - f(-2 * eps)) / (4 * eps)
        log.append((round(d1, 6), round(d2, 6)))
        return d1 if abs(d1 - d2) <= 1e-5 * max(1.0, abs(d1)) else None

    # directions supported on one replica (the others' terms cancel exactly
    # in the differences, so small steps stay far above round-off); a
    # direction whose interval moves a pair across r_c or r_d within the 50
    # steps (the forces have a kink there) is detected by two step sizes and
    # skipped
    checked = 0
    for r in (3, 17, 40, 58):
        a0, a1 = b.offsets[r], b.offsets[r + 1]
        dx = torch.zeros_like(x0)
        dx[a0:a1] = torch.tensor(rng.normal(size=(a1 - a0, 3)), device=dev)
        d = fd(lambda e: fwd(x0.detach() + e * dx, v0.detach()), 1e-8)
        if d is not None:
            assert abs(d - float((x0.grad * dx).sum())) <= 1e-3 * max(1.0, abs(d)), r
            checked += 1
        dv = torch.zeros_like(v0)
        dv[a0:a1] = torch.tensor(rng.normal(size=(a1 - a0, 3)), device=dev)
        d = fd(lambda e: fwd(x0.detach(), v0.detach() + e * dv), 1e-8)
        if d is not None:
            assert abs(d - float((v0.grad * dv).sum())) <= 1e-3 * max(1.0, abs(d)), r
            checked += 1
    for r in (0, 31, 63):
        for name, T in (("A", A), ("B", B)):
            E = torch.zeros_like(T)
            E[r, 0, 0] = 1.0

            def f(e, name=name, E=E):
                if name == "A":
                    return fwd(x0.detach(), v0.detach(), AA=A.detach() + e * E)
                return fwd(x0.detach(), v0.detach(), BB=B.detach() + e * E)
            d = fd(f, 1e-7)
            if d is not None:
                assert abs(d - float(T.grad[r, 0, 0])) <= 1e-3 * max(1.0, abs(d)), (r, name)
                checked += 1
    assert checked >= 8, log


def test_fit_A_B_to_target_density_and_surface_tension(env):
    """Batched calibration of (A, B) to a target density and surface tension.

    128 slab replicas of uneven size (1,000 to 2,500 particles) form four
    ensembles of 32; the replicas of an ensemble share one (A, B), and the
    four ensembles start at the corners of [-50, -30] x [15, 35].  An
    ensemble's observables are its replicas' mean local density (Sec. 2.1)
    and mean surface tension (L_x / 2)(P_xx - (P_yy + P_zz)/2) (Sec. 4.1, two
    interfaces) after a 20-step window; the targets are the same observables
    made with (A, B) = (-40, 25) from the same states and random streams.
    Levenberg-Marquardt, with both rows of each ensemble's 2 x 2 Jacobian
    from batched window gradients (one launch per kernel for all 128
    replicas), recovers (-40, 25) in every ensemble.  (One small slab's
    instantaneous surface tension is too noisy to fit on its own, and over
    much longer windows the trajectory's chaos makes the gradient of a single
    realisation rough: the ensemble mean over a short window is smooth.)"""
    torch, M, AD = env
    dev = "cuda"
    nrep, ngrp = 128, 4
    ws = _slab_batch(nrep, 33, n_range=(1000, 2500))
    ps = []
    for w in ws:
        p = w.params.copy()
        p.A[:] = -40.0
        p.B[:] = 25.0
        ps.append(p)
    b = M.Batch(ps, [w.n for w in ws], np.concatenate([w.pos for w in ws]),
                np.concatenate([w.vel for w in ws]), np.concatenate([w.type for w in ws]),
                [w.seed for w in ws])
    b.step(300)                            # slabs at (-40, 25)
    b.sync()
    xs, vs, _, _ = b.state()
    x0 = torch.tensor(xs, device=dev)
    v0 = torch.tensor(vs, device=dev)
    G = torch.tensor(np.stack([p.gamma for p in ps]), device=dev)
    ones = torch.ones((nrep, 8, 8), dtype=torch.float64, device=dev)
    vol = torch.tensor([float(np.prod(p.box)) for p in ps], device=dev)
    lx = torch.tensor([float(p.box[0]) for p in ps], device=dev)
    seg = torch.repeat_interleave(torch.arange(nrep, device=dev),
                                  torch.tensor(b.n_list, device=dev))
    counts = torch.tensor(b.n_list, dtype=torch.float64, device=dev)
    grp = torch.arange(nrep, device=dev) % ngrp
    K = 20

    def observables(theta_g):
        theta = theta_g[grp]
        A = theta[:, 0, None, None] * ones
        B = theta[:, 1, None, None] * ones
        xk, vk, rho, W = AD.window(b, ps, x0, v0, A, B, G, K, step0=300, observables=True)
        kin = torch.zeros((nrep, 3), dtype=torch.float64, device=dev).index_add_(0, seg, vk * vk)
        dens = torch.zeros(nrep, dtype=torch.float64, device=dev).index_add_(0, seg, rho) / counts
        P = (kin + W[:, :3]) / vol[:, None]
        gam = 0.5 * lx * (P[:, 0] - 0.5 * (P[:, 1] + P[:, 2]))
        per = float(nrep // ngrp)
        dg = torch.zeros(ngrp, dtype=torch.float64, device=dev).index_add_(0, grp, dens) / per
        gg = torch.zeros(ngrp, dtype=torch.float64, device=dev).index_add_(0, grp, gam) / per
        return dg, gg

    star = torch.tensor([[-40.0, 25.0]] * ngrp, dtype=torch.float64, device=dev)
    with torch.no_grad():
        d_t, g_t = observables(star)

    def residuals(th):
        dens, gam = observables(th)
        return torch.stack([(dens - d_t) / d_t, (gam - g_t) / 10.0], 1)

    # Levenberg-Marquardt per ensemble: a trial step is kept where it lowers
    # that ensemble's residual, else its damping grows
    theta = torch.tensor([[-46.0, 19.0], [-34.0, 31.0], [-46.0, 31.0], [-34.0, 19.0]],
                         dtype=torch.float64, device=dev)
    lam = torch.full((ngrp,), 1e-2, dtype=torch.float64, device=dev)
    hist = []
    for it in range(60):
        th = theta.clone().requires_grad_(True)
        res = residuals(th)
        J1 = torch.autograd.grad(res[:, 0].sum(), th, retain_graph=True)[0]
        J2 = torch.autograd.grad(res[:, 1].sum(), th)[0]
        J = torch.stack([J1, J2], 1)                                  # (ngrp, 2, 2)
        res = res.detach()
        f0 = (res ** 2).sum(1)
        hist.append(float(f0.max()))
        if hist[-1] < 1e-20:
            break
        JtJ = J.transpose(1, 2) @ J
        D = torch.diag_embed(torch.diagonal(JtJ, dim1=1, dim2=2))
        g = J.transpose(1, 2) @ res.unsqueeze(-1)
        step = torch.linalg.solve(JtJ + lam[:, None, None] * D, -g).squeeze(-1)
        trial = theta + step.clamp(-2.0, 2.0)                        # a trust region
        with torch.no_grad():
            f1 = (residuals(trial) ** 2).sum(1)
        ok = f1 < f0
        theta = torch.where(ok[:, None], trial, theta)
        lam = torch.where(ok, lam / 3.0, lam * 4.0).clamp(1e-12, 1e12)
    err = (theta - star).abs().cpu().numpy()
    assert err[:, 0].max() < 0.4 and err[:, 1].max() < 0.25, (theta.cpu().numpy(), it, hist)
