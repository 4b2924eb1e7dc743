"""Adjoint of the force evaluation and of velocity-Verlet windows on the GPU,
against the oracle's adjoint (itself pinned by finite differences) and against
central finite differences of the GPU forward."""
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


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-4)])
@pytest.mark.parametrize("frozen", [(), (1,)])
def test_force_vjp_matches_oracle(env, precision, tol, frozen):
    torch, M, AD = env
    w = I.tiny(1500, (6.0, 6.5, 5.5), 12, ntypes=2, frozen_types=frozen, g=(0.1, 0, 0))
    p = w.params.copy(precision=precision)
    s = M.System(p, w.pos, w.vel, w.type, w.seed)
    M.mdpd_set_step(s.h, 7)
    s.set_state(w.pos, w.vel)
    abar = np.random.default_rng(3).normal(size=w.pos.shape)
    xb, ub, tb = AD.force_vjp(s, torch.tensor(abar, device="cuda"))
    o = O.Oracle(p, w.pos, w.vel, w.type, w.seed, use_cells=True)
    oxb, oub, otb = o.force_vjp(abar, step=7)
    assert _rel(xb.cpu().numpy(), oxb) < tol
    assert _rel(ub.cpu().numpy(), oub) < tol
    for q in range(3):
        assert _rel(tb[q, :2, :2].cpu().numpy(), otb[q, :2, :2]) < tol * 10, q
    s.close()


def test_window_gradient_matches_oracle_and_finite_differences(env):
    torch, M, AD = env
    w = I.tiny(600, (4.5, 4.2, 4.8), 21, ntypes=2, g=(0.05, 0.0, 0.0))
    p = w.params.copy(precision=0)
    K = 8
    s = M.System(p, w.pos, w.vel, w.type, w.seed)
    dev = "cuda"
    x0 = torch.tensor(w.pos, device=dev, requires_grad=True)
    v0 = torch.tensor(w.vel, device=dev, requires_grad=True)
    A = torch.tensor(p.A, device=dev, requires_grad=True)
    B = torch.tensor(p.B, device=dev, requires_grad=True)
    G = torch.tensor(p.gamma, device=dev, requires_grad=True)
    rng = np.random.default_rng(5)
    cx = torch.tensor(rng.normal(size=w.pos.shape), device=dev)
    cv = torch.tensor(rng.normal(size=w.pos.shape), device=dev)
    xk, vk = AD.window(s, p, x0, v0, A, B, G, K, step0=3)
    loss = (cx * xk).sum() + (cv * vk).sum()
    loss.backward()
    # the oracle's chain rule on the same window
    o = O.Oracle(p, w.pos, w.vel, w.type, w.seed, use_cells=True)
    o.step = 3
    o.refresh()
    ck = OAD.window_forward(o, K)
    np.testing.assert_allclose(xk.detach().cpu().numpy(), o.x, atol=1e-11)
    oxb, ovb, otb = OAD.window_vjp(o, ck, cx.cpu().numpy(), cv.cpu().numpy())
    assert _rel(x0.grad.cpu().numpy(), oxb) < 1e-8
    assert _rel(v0.grad.cpu().numpy(), ovb) < 1e-8
    assert _rel(A.grad.cpu().numpy(), otb[0]) < 1e-8
    assert _rel(B.grad.cpu().numpy(), otb[1]) < 1e-8
    assert _rel(G.grad.cpu().numpy(), otb[2]) < 1e-8

    # central differences of the GPU forward (kink-free directions)
    def fwd(xx, vv, AA=A, BB=B, GG=G):
        with torch.no_grad():
            a, b = AD.window(s, p, xx, vv, AA, BB, GG, K, step0=3)
            return float((cx * a).sum() + (cv * b).sum())

    def fd(f, eps):
        d1 = (f(eps) - f(-eps)) / (2 * eps)
        d2 = (f(2 * eps) - f(-2 * eps)) / (4 * eps)
        return d1 if abs(d1 - d2) <= 1e-6 * max(1.0, abs(d1)) else None
    checked = 0
    for _ in range(3):
        dx = torch.tensor(rng.normal(size=w.pos.shape), device=dev)
        d = fd(lambda e: fwd(x0.detach() + e * dx, v0.detach()), 1e-7)
        if d is not None:
            assert abs(d - float((x0.grad * dx).sum())) <= 1e-3 * max(1.0, abs(d))
            checked += 1
        dv = torch.tensor(rng.normal(size=w.pos.shape), device=dev)
        d = fd(lambda e: fwd(x0.detach(), v0.detach() + e * dv), 1e-7)
        if d is not None:
            assert abs(d - float((v0.grad * dv).sum())) <= 1e-3 * max(1.0, abs(d))
            checked += 1
    for name, T in (("A", A), ("B", B), ("G", G)):
        E = torch.zeros_like(T)
        E[0, 1] = E[1, 0] = 1.0

        def f(e, name=name, E=E):
            kw = {"AA": A.detach(), "BB": B.detach(), "GG": G.detach()}
            kw["AA" if name == "A" else "BB" if name == "B" else "GG"] = T.detach() + e * E
            return fwd(x0.detach(), v0.detach(), **kw)
        d = fd(f, 1e-6)
        if d is not None:
            assert abs(d - float(T.grad[0, 1])) <= 1e-3 * max(1.0, abs(d)), (name, d, T.grad[0, 1])
            checked += 1
    assert checked >= 4
    s.close()


def test_fit_A_B_from_a_target_window(env):
    """The adjoint drives a fit: from a 10-step window generated with
    (A, B) = (-40, 25), L-BFGS on |x_K - x_K*|^2 + |v_K - v_K*|^2 with the
    window gradient recovers A and B when started from (-34, 20)."""
    torch, M, AD = env
    w = I.tiny(500, (4.5, 4.5, 4.5), 31)
    p = w.params.copy(precision=0)
    s = M.System(p, w.pos, w.vel, w.type, w.seed)
    dev = "cuda"
    x0 = torch.tensor(w.pos, device=dev)
    v0 = torch.tensor(w.vel, device=dev)
    G = torch.tensor(p.gamma, device=dev)
    K = 10
    with torch.no_grad():
        xt, vt = AD.window(s, p, x0, v0, torch.tensor(p.A, device=dev),
                           torch.tensor(p.B, device=dev), G, K)
    theta = torch.tensor([-34.0, 20.0], dtype=torch.float64, device=dev, requires_grad=True)
    ones = torch.ones((8, 8), dtype=torch.float64, device=dev)
    opt = torch.optim.LBFGS([theta], lr=1.0, max_iter=60, tolerance_grad=1e-12,
                            tolerance_change=1e-14, line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        xk, vk = AD.window(s, p, x0, v0, theta[0] * ones, theta[1] * ones, G, K)
        loss = ((xk - xt) ** 2).sum() + ((vk - vt) ** 2).sum()
        loss.backward()
        return loss

    opt.step(closure)
    a, b = theta.detach().cpu().numpy()
    assert abs(a - (-40.0)) < 1e-3 * 40 and abs(b - 25.0) < 1e-3 * 25, (a, b)
    s.close()


def _oracle_density_loss(w, p, x, rb):
    o = O.Oracle(p, x, w.vel, w.type, w.seed, use_cells=True)
    return float(np.sum(rb * o.density()))


@pytest.mark.parametrize("frozen", [(), (1,)])
def test_density_vjp_matches_oracle_finite_differences(env, frozen):
    """d(sum_i rhobar_i rho_i)/dx from the density pass's VJP kernel against
    central differences of the oracle's densities (FP64; w_rho is C1 at r_d,
    so the differences have no kink)."""
    torch, M, AD = env
    w = I.tiny(900, (5.0, 5.5, 4.5), 23, ntypes=2, frozen_types=frozen)
    p = w.params.copy(precision=0)
    s = M.System(p, w.pos, w.vel, w.type, w.seed)
    rng = np.random.default_rng(5)
    rb = rng.normal(size=w.n)
    x = torch.tensor(w.pos, device="cuda")
    xt = x.clone().requires_grad_(True)
    rho = AD.density(s, xt)
    assert np.allclose(rho.detach().cpu().numpy(),
                       O.Oracle(p, w.pos, w.vel, w.type, w.seed).density(), rtol=1e-13, atol=1e-13)
    (rho * torch.tensor(rb, device="cuda")).sum().backward()
    g = xt.grad.cpu().numpy()
    eps = 1e-6
    for _ in range(3):
        d = rng.normal(size=w.pos.shape)
        fd = (_oracle_density_loss(w, p, w.pos + eps * d, rb) -
              _oracle_density_loss(w, p, w.pos - eps * d, rb)) / (2 * eps)
        assert abs(fd - np.sum(g * d)) <= 1e-6 * max(1.0, abs(fd)), (fd, np.sum(g * d))
    s.close()


def test_fit_A_to_a_target_local_density(env):
    """Calibration through the window and the density VJP: the mean local
    density after a 10-step window of a bulk box is the target made with
    A = -40 (B fixed at 25); gradient descent on A from -30 on
    (mean rho(x_K) - target)^2 approaches -40."""
    torch, M, AD = env
    w = I.tiny(700, (5.0, 5.0, 5.0), 41)
    p = w.params.copy(precision=0)
    s = M.System(p, w.pos, w.vel, w.type, w.seed)
    dev = "cuda"
    x0 = torch.tensor(w.pos, device=dev)
    v0 = torch.tensor(w.vel, device=dev)
    ones = torch.ones((8, 8), dtype=torch.float64, device=dev)
    B = torch.tensor(p.B, device=dev)
    G = torch.tensor(p.gamma, device=dev)
    K = 10
    with torch.no_grad():
        xt, _ = AD.window(s, p, x0, v0, -40.0 * ones, B, G, K)
    target = float(AD.density(s, xt).mean())

    def loss_and_grad(a):
        A = torch.tensor(a, dtype=torch.float64, device=dev, requires_grad=True)
        xk, _ = AD.window(s, p, x0, v0, A * ones, B, G, K)
        # the density op sets the state in between: the window's checkpoints
        # are not disturbed by that
        loss = (AD.density(s, xk).mean() - target) ** 2
        loss.backward()
        return float(loss.detach()), float(A.grad)

    a = -30.0
    l0, _ = loss_and_grad(a)
    for _ in range(12):
        l, g = loss_and_grad(a)
        # Newton-like step on the scalar quadratic model l = (m(a) - t)^2
        step = 2.0 * l / g if g != 0 else 0.0
        a -= float(np.clip(step, -5.0, 5.0))
    lf, _ = loss_and_grad(a)
    assert lf < 1e-3 * l0, (l0, lf, a)
    assert abs(a - (-40.0)) < 0.5, a
    s.close()
