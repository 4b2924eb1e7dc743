"""Statistical checks at the configurations' own sizes and parameters.

The oracle cannot run these to length on the host, so the GPU's FP32 path is
checked against its FP64 path (itself pinned to the oracle step by step) and
against what the physics fixes:

* liquid-vapour slab, 60 x 20 x 20 box, 48,000 particles (Sec. 4.1 shape):
  the interior density is the coexistence density, the zero of the Fig. 3b
  equation of state; the surface tension (L_x / 2) <P_xx - (P_yy + P_zz)/2>
  agrees between FP32 and FP64;
* slit pore, 100 x 40 periodic, channel height 20 between frozen walls at
  density 6 (A_fs = -30), body force 0.02 (the Poiseuille set-up): the time
  averaged u_x(z) is a parabola and FP32 and FP64 give the same viscosity;
* synthetic rock, 256^3 voxels (Sec. 5-6 stand-in): the superficial flux q
  is resolved at three driving forces and the effective permeability
  k(g) = eta q / (rho g) is reported with eta from the slit, with the
  exponent of q ~ g^a.  The paper finds the flow rate in shale nanopores
  deviating from Darcy's law (a non-constant permeability, Sec. 6); here too
  q grows faster than g.  At the rock's own g = 0.01 the flux (about 1e-4)
  is below the thermal noise of the fluid's total momentum (about 6e-4 per
  decorrelated sample of 1.9M particles), so the forces are 0.1, 0.2, 0.4
  (pore Reynolds number at most about 0.1).
"""
import math
import os

import numpy as np
import pytest

from paper_1903_10134_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10134_gb300 import mdpd
    mdpd.lib()
    return mdpd


def block_stats(samples, nblocks=8):
    a = np.asarray(samples, dtype=float)
    bm = np.array([b.mean(axis=0) for b in np.array_split(a, nblocks)])
    return a.mean(axis=0), bm.std(axis=0, ddof=1) / math.sqrt(nblocks)


def eos_zero(golden_dir):
    """Coexistence density of the Fig. 3b equation of state (its zero above
    rho = 3), by bisection."""
    g = {}
    for line in open(os.path.join(golden_dir, "eos.txt")):
        f = line.split()
        if len(f) == 2 and not line.startswith("#"):
            g[f[0]] = float(f[1])

    def p(rho):
        a = g["mdpd_alpha"]
        return (rho + a * g["mdpd_A"] * rho ** 2 +
                2 * a * g["mdpd_B"] * g["mdpd_rd"] ** 4 *
                (rho ** 3 - g["mdpd_c"] * rho ** 2 + g["mdpd_d"]))
    lo, hi = 3.0, 9.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if (p(lo) < 0) == (p(mid) < 0):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_full_slab_coexistence_density_and_surface_tension(M, golden_dir):
    w = I.slab(seed=11, precision=1)              # 60 x 20 x 20, N = 48,000
    Lx, Ly, Lz = w.params.box
    V = Lx * Ly * Lz
    nb = 30
    res = {}
    for prec in (1, 0):
        s = M.System(w.params.copy(precision=prec), w.pos, w.vel, w.type, w.seed)
        s.step(5000)                              # 50 time units: the slab forms
        prof, gam = [], []
        for k in range(100):
            for _ in range(10):
                s.step(20)
                o = s.observables()
                P = (o[11:14] + o[5:8]) / V
                gam.append(0.5 * Lx * (P[0] - 0.5 * (P[1] + P[2])))
            x = s.state()[0][:, 0]
            th = 2 * np.pi * x / Lx
            com = Lx / (2 * np.pi) * np.arctan2(np.sin(th).mean(), np.cos(th).mean())
            h, _ = np.histogram((x - com + Lx / 2) % Lx, bins=nb, range=(0, Lx))
            prof.append(h / (Lx / nb * Ly * Lz))
        s.close()
        pm, pe = block_stats(prof)
        gm, ge = block_stats(gam)
        interior = block_stats(np.asarray(prof)[:, nb // 2 - 3: nb // 2 + 3].mean(1))
        res[prec] = (pm, pe, gm, ge, interior)
        print("full slab", "fp32" if prec else "fp64", "interior %.4f +- %.4f" % interior,
              "gamma %.3f +- %.3f" % (gm, ge))
    rho_eos = eos_zero(golden_dir)
    for prec in (1, 0):
        dens, err = res[prec][4]
        assert abs(dens - rho_eos) < 0.05, (prec, dens, rho_eos)
    # FP32 against FP64: surface tension within 3 combined standard errors,
    # the interior density within 3 sigma plus 0.005
    g32, e32, g64, e64 = res[1][2], res[1][3], res[0][2], res[0][3]
    assert abs(g32 - g64) <= 3 * math.hypot(e32, e64), (g32, e32, g64, e64)
    d32, s32 = res[1][4]
    d64, s64 = res[0][4]
    assert abs(d32 - d64) <= 3 * math.hypot(s32, s64) + 0.005, (d32, d64)
    # a physical slab: positive surface tension
    assert g32 > 4 * e32


def _profile(x, v, nf, H, nb):
    z = x[:nf, 2]
    idx = np.clip((z / H * nb).astype(int), 0, nb - 1)
    return np.bincount(idx, weights=v[:nf, 0], minlength=nb) / np.maximum(
        np.bincount(idx, minlength=nb), 1)


@pytest.fixture(scope="module")
def slit_viscosity(M):
    """The full-size slit (Poiseuille set-up): FP32 develops the flow from
    rest (about three decay times of the slowest mode, H^2 / (pi^2 nu)), then
    FP32 and an FP64 handle made from the same developed state each average
    the u_x(z) profile; returns per precision (profile, error, fitted eta,
    R^2) and the fluid density."""
    w = I.slit(seed=5, precision=1)               # 100 x 40, H = 20, g = 0.02
    H, g, nf = 20.0, w.params.g[0], w.n
    Lx, Ly = w.params.box[0], w.params.box[1]
    rho = nf / (Lx * Ly * H)
    nb = 20
    s32 = M.System.from_workload(w)
    s32.step(20000)
    x, v, t, _ = s32.state()
    p64 = w.params.copy(precision=0)
    s64 = M.System(p64, x, v, t, w.seed)
    # the wall particles are already in the state: the mask only (no packing)
    s64.set_walls(w.mask, w.voxel, w.origin, 0.0, w.shell, w.wall_type, w.wall_seed)
    M.mdpd_set_step(s64.h, M.mdpd_step_count(s32.h))
    out = {}
    zc = (np.arange(nb) + 0.5) * H / nb
    for name, s in (("fp32", s32), ("fp64", s64)):
        prof = []
        for _ in range(30):
            s.step(200)
            xs, vs, _, _ = s.state()
            prof.append(_profile(xs, vs, nf, H, nb))
        s.close()
        m, e = block_stats(prof, nblocks=6)
        Aq = np.stack([zc * (H - zc), np.ones_like(zc)], 1)
        coef, *_ = np.linalg.lstsq(Aq, m, rcond=None)
        pred = Aq @ coef
        r2 = 1 - np.sum((m - pred) ** 2) / np.sum((m - m.mean()) ** 2)
        eta = rho * g / (2 * coef[0])             # u = (rho g / 2 eta) z (H - z) + u_s
        out[name] = (m, e, eta, r2, coef[1])
        print("full slit", name, "eta %.4f" % eta, "R2 %.5f" % r2, "slip %.4f" % coef[1],
              np.round(m, 4).tolist())
    return out, rho


def test_full_slit_poiseuille_parabola_and_viscosity(slit_viscosity):
    out, rho = slit_viscosity
    for name in ("fp32", "fp64"):
        m, e, eta, r2, slip = out[name]
        assert r2 > 0.99, (name, r2)
        assert eta > 0
    e32, e64 = out["fp32"][2], out["fp64"][2]
    assert abs(e32 - e64) <= 0.03 * e64, (e32, e64)


def test_full_rock_flux_and_effective_permeability(M, slit_viscosity):
    """256^3-voxel rock (4.36M particles, porosity 0.15): the superficial
    velocity q = sum_fluid v_x / V_box (block means of the library's running
    observable averages) is resolved at g = 0.1, 0.2, 0.4 and grows with g;
    k(g) = eta q / (rho g) and the exponent of q ~ g^a are reported."""
    out, _ = slit_viscosity
    eta = out["fp32"][2]
    res = {}
    for g in (0.1, 0.2, 0.4):
        w = I.rock(g=g, seed=1, precision=1)
        s = M.System.from_workload(w)
        nf = w.n
        V = float(np.prod(w.params.box))
        rho = nf / (V * 0.15)                     # fluid density in the pores
        s.step(1500)
        s.observables_mean(reset=True)
        qs = []
        for _ in range(12):
            s.step(500)
            qs.append(s.observables_mean(reset=True)[0] / V)   # mobile = fluid momentum
        s.close()
        q, qe = block_stats(qs, nblocks=6)
        res[g] = (q, qe, eta * q / (rho * g))
        print("full rock g=%.2f q %.6f +- %.6f  k %.6f (eta %.4f rho %.4f)"
              % (g, q, qe, res[g][2], eta, rho))
    gs = np.array(sorted(res))
    qv = np.array([res[g][0] for g in gs])
    a = np.polyfit(np.log(gs), np.log(qv), 1)[0]
    print("full rock q ~ g^%.3f" % a)
    for g in (0.2, 0.4):
        assert res[g][0] > 5 * res[g][1], (g, res[g])        # the flux is resolved
    assert qv[0] < qv[1] < qv[2], qv
    assert all(res[g][2] > 0 for g in gs)
