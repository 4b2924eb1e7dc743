"""Pins of the oracle's vector-Jacobian product of one force evaluation against
central finite differences of the oracle's own forward forces (FP64).

L(x, u, theta) = sum_i abar_i . a_i with the random stream of one step held
fixed; the VJP must give dL/dx, dL/du and dL/d(A, B, gamma) (symmetric
per-type-pair parameters).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_10134_gb300 import inputs as I


def _system(n=120, L=(3.6, 3.4, 3.8), seed=3, ntypes=2, frozen=()):
    w = I.tiny(n, L, seed, ntypes=ntypes, frozen_types=frozen)
    return w


def _loss(o, abar, x=None, u=None, params=None, step=5):
    if params is not None:
        o.sys, o._mask = O.make_sys(params, o.sys.seed, bool(o.sys.use_cells))
    a, _ = o.forces(x=x, v=u, step=step)
    return float(np.sum(abar * a))


@pytest.mark.parametrize("frozen", [(), (1,)])
def test_force_vjp_matches_finite_differences(frozen):
    w = _system(frozen=frozen)
    o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed)
    rng = np.random.default_rng(1)
    abar = rng.normal(size=w.pos.shape)
    xb, ub, tb = o.force_vjp(abar, step=5)
    eps = 1e-6
    for _ in range(3):
        dx = rng.normal(size=w.pos.shape)
        fd = (_loss(o, abar, x=w.pos + eps * dx) - _loss(o, abar, x=w.pos - eps * dx)) / (2 * eps)
        assert abs(fd - np.sum(xb * dx)) <= 1e-5 * max(1.0, abs(fd)), (fd, np.sum(xb * dx))
        du = rng.normal(size=w.pos.shape)
        fd = (_loss(o, abar, u=w.vel + eps * du) - _loss(o, abar, u=w.vel - eps * du)) / (2 * eps)
        assert abs(fd - np.sum(ub * du)) <= 1e-6 * max(1.0, abs(fd))
    base = w.params
    for q, name in enumerate(("A", "B", "gamma")):
        for (a, b) in ((0, 0), (0, 1), (1, 1)):
            pp, pm = base.copy(), base.copy()
            for p_, sgn in ((pp, 1), (pm, -1)):
                tab = getattr(p_, name)
                tab[a, b] += sgn * eps
                if a != b:
                    tab[b, a] += sgn * eps
            fd = (_loss(o, abar, params=pp) - _loss(o, abar, params=pm)) / (2 * eps)
            o.sys, o._mask = O.make_sys(base, o.sys.seed, bool(o.sys.use_cells))
            assert abs(fd - tb[q, a, b]) <= 1e-5 * max(1.0, abs(fd)), (name, a, b, fd, tb[q, a, b])
            assert tb[q, a, b] == tb[q, b, a]


def test_force_vjp_of_pure_translation_is_zero():
    """Translating every particle leaves all forces unchanged, so the position
    adjoint sums to zero over particles (no frozen particles)."""
    w = _system()
    o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed)
    abar = np.random.default_rng(2).normal(size=w.pos.shape)
    xb, ub, _ = o.force_vjp(abar)
    scale = np.abs(xb).max()
    assert np.abs(xb.sum(axis=0)).max() < 1e-11 * scale * w.n
    # a uniform velocity shift does not change u_ij either
    assert np.abs(ub.sum(axis=0)).max() < 1e-11 * np.abs(ub).max() * w.n


def _window_loss(w, params, x0, v0, K, cx, cv):
    o = O.Oracle(params, x0, v0, w.type, w.seed)
    o.run(K)
    return float(np.sum(cx * o.x) + np.sum(cv * o.v))


def _fd(f, eps):
    """Central difference at eps and 2 eps; None if they disagree (a pair crossed
    r_c or r_d inside the interval, where the forces have a kink)."""
    d1 = (f(eps) - f(-eps)) / (2 * eps)
    d2 = (f(2 * eps) - f(-2 * eps)) / (4 * eps)
    return d1 if abs(d1 - d2) <= 1e-6 * max(1.0, abs(d1)) else None


@pytest.mark.parametrize("frozen", [(), (1,)])
def test_window_gradient_matches_finite_differences(frozen):
    """Chain rule through a 6-step velocity-Verlet window against central
    differences of whole oracle trajectories (the random stream is fixed by
    the step index).  Directions whose difference interval contains a cutoff
    crossing are skipped; most are kink-free."""
    from oracle import adjoint as AD
    w = _system(n=90, L=(3.3, 3.5, 3.4), seed=8, frozen=frozen)
    K = 6
    rng = np.random.default_rng(4)
    cx = rng.normal(size=w.pos.shape)
    cv = rng.normal(size=w.pos.shape)
    o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed)
    ck = AD.window_forward(o, K)
    xb, vb, tb = AD.window_vjp(o, ck, cx, cv)
    eps = 1e-7
    checked = 0
    for _ in range(4):
        dx = rng.normal(size=w.pos.shape)
        fd = _fd(lambda e: _window_loss(w, w.params, w.pos + e * dx, w.vel, K, cx, cv), eps)
        if fd is not None:
            assert abs(fd - np.sum(xb * dx)) <= 1e-4 * max(1.0, abs(fd)), (fd, np.sum(xb * dx))
            checked += 1
        dv = rng.normal(size=w.pos.shape)
        fd = _fd(lambda e: _window_loss(w, w.params, w.pos, w.vel + e * dv, K, cx, cv), eps)
        if fd is not None:
            assert abs(fd - np.sum(vb * dv)) <= 1e-4 * max(1.0, abs(fd)), (fd, np.sum(vb * dv))
            checked += 1
    assert checked >= 4
    for q, name in enumerate(("A", "B", "gamma")):
        a, b = (0, 1)

        def f(e, name=name):
            p_ = w.params.copy()
            tab = getattr(p_, name)
            tab[a, b] += e
            tab[b, a] += e
            return _window_loss(w, p_, w.pos, w.vel, K, cx, cv)
        fd = _fd(f, 1e-6)
        if fd is not None:
            assert abs(fd - tb[q, a, b]) <= 1e-4 * max(1.0, abs(fd)), (name, fd, tb[q, a, b])


def _obs_loss(o, cvir, rb, x=None, params=None, step=5):
    """sum_k cvir_k W_k + sum_i rb_i rho_i of one oracle evaluation (the
    conservative virial of the pressure tensor, Sec. 4.1, and the local
    densities of Sec. 2.1)."""
    if params is not None:
        o.sys, o._mask = O.make_sys(params, o.sys.seed, bool(o.sys.use_cells))
    _, vir = o.forces(x=x, step=step)
    return float(np.sum(cvir * vir) + np.sum(rb * o.density(x)))


@pytest.mark.parametrize("frozen", [(), (1,)])
def test_virial_and_density_vjp_match_finite_differences(frozen):
    """The virial and density cotangents of the oracle's evaluation VJP
    against central differences of its own virial and densities: positions
    and A, B move them; velocities and gamma do not."""
    w = _system(frozen=frozen)
    o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed)
    rng = np.random.default_rng(11)
    cvir = rng.normal(size=6)
    rb = rng.normal(size=w.n)
    xb, ub, tb = o.eval_vjp(None, cvir, rb, step=5)
    assert np.all(ub == 0.0) and np.all(tb[2] == 0.0)
    eps = 1e-6
    for _ in range(3):
        dx = rng.normal(size=w.pos.shape)
        fd = (_obs_loss(o, cvir, rb, x=w.pos + eps * dx) -
              _obs_loss(o, cvir, rb, x=w.pos - eps * dx)) / (2 * eps)
        assert abs(fd - np.sum(xb * dx)) <= 1e-5 * max(1.0, abs(fd)), (fd, np.sum(xb * dx))
    base = w.params
    for q, name in enumerate(("A", "B")):
        for (a, b) in ((0, 0), (0, 1), (1, 1)):
            pp, pm = base.copy(), base.copy()
            for p_, sgn in ((pp, 1), (pm, -1)):
                tab = getattr(p_, name)
                tab[a, b] += sgn * eps
                if a != b:
                    tab[b, a] += sgn * eps
            fd = (_obs_loss(o, cvir, rb, params=pp) - _obs_loss(o, cvir, rb, params=pm)) / (2 * eps)
            o.sys, o._mask = O.make_sys(base, o.sys.seed, bool(o.sys.use_cells))
            assert abs(fd - tb[q, a, b]) <= 1e-5 * max(1.0, abs(fd)), (name, a, b, fd, tb[q, a, b])


def test_eval_vjp_is_linear_in_its_cotangents():
    """The evaluation VJP with all three cotangents is the sum of the three
    taken one at a time (each term is added separately by the chain rule)."""
    w = _system(ntypes=2, frozen=(1,))
    o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed)
    rng = np.random.default_rng(12)
    ab, cv, rb = rng.normal(size=w.pos.shape), rng.normal(size=6), rng.normal(size=w.n)
    full = o.eval_vjp(ab, cv, rb, step=5)
    parts = [o.eval_vjp(ab, None, None, step=5), o.eval_vjp(None, cv, None, step=5),
             o.eval_vjp(None, None, rb, step=5)]
    for k in range(3):
        np.testing.assert_allclose(full[k], sum(p[k] for p in parts), rtol=1e-12,
                                   atol=1e-12 * max(1.0, np.abs(full[k]).max()))
    np.testing.assert_array_equal(parts[0][0], o.force_vjp(ab, step=5)[0])


def test_window_gradient_with_final_observables_matches_finite_differences():
    """A window loss on the final positions and velocities plus the last
    evaluation's virial and densities (what a fit to a target density and
    surface tension differentiates), against central differences of whole
    oracle trajectories."""
    from oracle import adjoint as AD
    w = _system(n=90, L=(3.3, 3.5, 3.4), seed=9)
    K = 5
    rng = np.random.default_rng(13)
    cx = rng.normal(size=w.pos.shape)
    cv = rng.normal(size=w.pos.shape)
    cvir = rng.normal(size=6)
    rb = rng.normal(size=w.n)

    def loss(params, x0, v0):
        o = O.Oracle(params, x0, v0, w.type, w.seed)
        o.run(K)
        return float(np.sum(cx * o.x) + np.sum(cv * o.v) + np.sum(cvir * o.virial) +
                     np.sum(rb * o.rho))

    o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed)
    ck = AD.window_forward(o, K)
    xb, vb, tb = AD.window_vjp(o, ck, cx, cv, cvir=cvir, rhobar=rb)
    checked = 0
    for _ in range(4):
        dx = rng.normal(size=w.pos.shape)
        fd = _fd(lambda e: loss(w.params, w.pos + e * dx, w.vel), 1e-7)
        if fd is not None:
            assert abs(fd - np.sum(xb * dx)) <= 1e-4 * max(1.0, abs(fd)), (fd, np.sum(xb * dx))
            checked += 1
    for q, name in enumerate(("A", "B")):
        def f(e, name=name):
            p_ = w.params.copy()
            getattr(p_, name)[0, 0] += e
            return loss(p_, w.pos, w.vel)
        fd = _fd(f, 1e-6)
        if fd is not None:
            assert abs(fd - tb[q, 0, 0]) <= 1e-4 * max(1.0, abs(fd)), (name, fd, tb[q, 0, 0])
            checked += 1
    assert checked >= 3
