"""Statistical parity of the CUDA library with the FP64 oracle on small
versions of the paper-shaped workloads (slab, slit pore, porous rock).

After a few hundred steps the trajectories of two implementations separate
(the dynamics is chaotic), so they are compared as independent samples of the
same ensemble: time averages with standard errors from block averages, and a
difference within 4 combined standard errors (plus a small allowance stated at
each check).  Three runs are compared: GPU FP32 pair arithmetic, GPU FP64, and
the oracle.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
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
    """Mean and standard error of a time series from block averages."""
    a = np.asarray(samples, dtype=float)
    blocks = np.array_split(a, nblocks)
    bm = np.array([b.mean(axis=0) for b in blocks])
    return a.mean(axis=0), bm.std(axis=0, ddof=1) / math.sqrt(nblocks)


def agree(m1, e1, m2, e2, allow=0.0):
    return np.all(np.abs(m1 - m2) <= 4.0 * np.hypot(e1, e2) + allow)


class GpuRun:
    def __init__(self, M, w, precision):
        p = w.params.copy(precision=precision)
        self.s = M.System(p, w.pos, w.vel, w.type, w.seed)
        if w.mask is not None:
            self.s.set_walls(w.mask, w.voxel, w.origin, w.wall_density, w.shell, w.wall_type,
                             w.wall_seed)

    def advance(self, k):
        self.s.step(k)

    def positions(self):
        return self.s.state()[0]

    def velocities(self):
        return self.s.state()[1]

    def obs(self):
        return self.s.observables()

    def close(self):
        self.s.close()


class OracleRun:
    def __init__(self, w):
        pos, vel, typ = w.pos, w.vel, w.type
        kw = {}
        if w.mask is not None:
            wpos, _ = O.place_walls(w.mask, w.params.periodic, w.voxel, w.origin,
                                    w.wall_density, w.shell, w.wall_seed)
            pos = np.concatenate([pos, wpos])
            vel = np.concatenate([vel, np.zeros_like(wpos)])
            typ = np.concatenate([typ, np.full(len(wpos), w.wall_type, np.int32)])
            kw = dict(mask=w.mask, voxel=w.voxel, origin=w.origin)
        self.o = O.Oracle(w.params.copy(precision=0), pos, vel, typ, w.seed, use_cells=True, **kw)
        self.last = None

    def advance(self, k):
        self.last, _ = self.o.run(k)

    def positions(self):
        return self.o.x

    def velocities(self):
        return self.o.v

    def obs(self):
        return self.last

    def close(self):
        pass


def run_all(M, w, equil, nsamp, every, sample):
    out = {}
    for name, mk in (("fp32", lambda: GpuRun(M, w, 1)), ("fp64", lambda: GpuRun(M, w, 0)),
                     ("oracle", lambda: OracleRun(w))):
        r = mk()
        r.advance(equil)
        vals = []
        for _ in range(nsamp):
            r.advance(every)
            vals.append(sample(r))
        r.close()
        out[name] = block_stats(vals)
    return out


def test_slab_density_profile_and_surface_tension(M):
    """Liquid-vapour slab (Sec. 4.1 shape): density profile along x, liquid
    density at the centre and surface tension from the pressure tensor,
    gamma = (L_x/2) <P_xx - (P_yy + P_zz)/2>."""
    Lx, Ly, Lz = 24.0, 8.0, 8.0
    w = I.slab(box=(Lx, Ly, Lz), slab_x=(8.0, 16.0), seed=7, precision=0, fill="lattice")
    nbins = 12
    V = Lx * Ly * Lz

    def sample(r):
        x = r.positions()[:, 0]
        th = 2 * np.pi * x / Lx                    # centre of mass on the periodic axis
        com = Lx / (2 * np.pi) * np.arctan2(np.sin(th).mean(), np.cos(th).mean())
        h, _ = np.histogram((x - com + Lx / 2) % Lx, bins=nbins, range=(0, Lx))
        dens = h / (Lx / nbins * Ly * Lz)
        o = r.obs()
        P = (o[11:14] + o[5:8]) / V
        gam = 0.5 * Lx * (P[0] - 0.5 * (P[1] + P[2]))
        return np.concatenate([dens, [gam, o[4]]])

    res = run_all(M, w, equil=400, nsamp=64, every=25, sample=sample)
    for k, (m, e) in res.items():
        print("slab", k, np.round(m, 3).tolist(), np.round(e, 3).tolist())
    for name in ("fp32", "fp64"):
        m, e = res[name]
        mo, eo = res["oracle"]
        # profile (all bins), surface tension, temperature
        assert agree(m[:nbins], e[:nbins], mo[:nbins], eo[:nbins], allow=0.15), (name, m, mo)
        assert agree(m[nbins], e[nbins], mo[nbins], eo[nbins], allow=0.3), (name, m[nbins], mo[nbins])
        # kT: GPU and oracle agree; the slab is a few time units past a random start,
        # so the level is checked loosely here (the +-2 % check is on a bulk run)
        assert agree(m[nbins + 1], e[nbins + 1], mo[nbins + 1], eo[nbins + 1], allow=0.005)
        assert abs(m[nbins + 1] - 1.0) < 0.06
    # the slab's interior sits at the coexistence density: the zero of the Fig. 3b
    # equation of state, rho = 6.10
    for name in ("fp32", "fp64", "oracle"):
        centre = res[name][0][nbins // 2 - 2: nbins // 2 + 2].mean()
        assert abs(centre - 6.10) < 0.15, (name, centre)


def test_slit_poiseuille_profile(M):
    """Slit pore with frozen walls and reflection, body force along x: the time
    averaged u_x(z) of the fluid is a parabola (R^2 > 0.97), and the GPU runs
    and the oracle agree on the profile and on the fitted viscosity."""
    H = 6.0
    w = I.slit(Lx=6.0, Ly=6.0, H=H, wall=1.0, voxel=0.5, g=0.2, seed=3, precision=0)
    nb = 6
    nf = w.n

    def sample(r):
        x = r.positions()[:nf]
        v = r.velocities()[:nf]
        z = x[:, 2]
        idx = np.clip((z / H * nb).astype(int), 0, nb - 1)
        u = np.array([v[idx == b, 0].mean() if np.any(idx == b) else 0.0 for b in range(nb)])
        return u

    res = run_all(M, w, equil=2000, nsamp=40, every=50, sample=sample)
    for k, (m, e) in res.items():
        print("slit", k, np.round(m, 4).tolist(), np.round(e, 4).tolist())
    zc = (np.arange(nb) + 0.5) * H / nb
    fits = {}
    for name, (m, e) in res.items():
        # u(z) = (rho g / 2 eta) z (H - z) + u_s  (u_s: slip)
        Aq = np.stack([zc * (H - zc), np.ones_like(zc)], 1)
        coef, *_ = np.linalg.lstsq(Aq, m, rcond=None)
        pred = Aq @ coef
        r2 = 1 - np.sum((m - pred) ** 2) / np.sum((m - m.mean()) ** 2)
        assert r2 > 0.97, (name, r2, m)
        fits[name] = coef[0]
    mo, eo = res["oracle"]
    for name in ("fp32", "fp64"):
        m, e = res[name]
        assert agree(m, e, mo, eo, allow=0.02), (name, m, mo)
        assert abs(fits[name] - fits["oracle"]) < 0.2 * abs(fits["oracle"]), fits


def test_small_rock_mean_flow(M):
    """Porous rock from a Gaussian random field (32^3 voxels at porosity 0.3),
    body force along x: the mean fluid velocity (the Darcy flux per fluid
    particle), the fluid density near walls and kT agree between GPU and oracle."""
    w = I.rock(nvox=32, voxel=0.5, corr=4.0, porosity=0.3, g=0.5, seed=5, precision=0)
    nf = w.n

    def sample(r):
        v = r.velocities()[:nf]
        return np.array([v[:, 0].mean(), v[:, 1].mean(), (v ** 2).sum(1).mean() / 3])

    res = run_all(M, w, equil=600, nsamp=32, every=25, sample=sample)
    for k, (m, e) in res.items():
        print("rock", k, np.round(m, 5).tolist(), np.round(e, 5).tolist())
    mo, eo = res["oracle"]
    assert mo[0] > 4 * eo[0]                      # the flow is resolved
    for name in ("fp32", "fp64"):
        m, e = res[name]
        assert agree(m, e, mo, eo, allow=0.003), (name, m, e, mo, eo)
        assert abs(m[2] - 1.0) < 0.06


def test_bulk_temperature_held(M):
    """The pairwise thermostat holds kT at the set value (sigma^2 = 2 gamma kT,
    Sec. 2.1): bulk mDPD liquid (Fig. 3 parameters), FP32 and FP64, 2 %."""
    w = I.bulk(n=6000, seed=9, precision=1)
    for prec in (1, 0):
        r = GpuRun(M, w, prec)
        r.advance(500)
        r.s.observables_mean(reset=True)
        r.advance(2000)
        kt = r.s.observables_mean()[4]
        r.close()
        assert abs(kt - 1.0) < 0.02, (prec, kt)
