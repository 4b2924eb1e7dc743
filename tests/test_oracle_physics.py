"""Physics pins of the oracle: the equilibrium its dynamics reach.

A thermostat obeying the fluctuation-dissipation theorem (Sec. 2.1 of
arXiv:1903.10134) samples exp(-U/kT); the mDPD conservative force (Eq. 1) is
the gradient of Warren's many-body potential.  So the oracle's time-averaged
virial pressure must match a Metropolis Monte Carlo of that potential
(tests/mc_reference.py, no shared code), and its temperature must be kT.
The paper's printed equations of state (Fig. 3 caption, tests/golden/eos.txt)
are fits; they are checked within the fits' quality.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_10134_gb300 import inputs as I
from tests.mc_reference import mc_pressure


def _golden(golden_dir):
    vals = {}
    with open(os.path.join(golden_dir, "eos.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _dpd_pressure(A, B, rho, L, seed=3, equil=300, blocks=10, block=200):
    n = int(round(rho * L ** 3))
    w = I.bulk(n, L=(L, L, L), seed=seed)
    w.params.A[:] = A
    w.params.B[:] = B
    o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed)
    o.run(equil)
    ps, kts = [], []
    for _ in range(blocks):
        _, mean = o.run(block)
        ps.append((mean[11] + mean[12] + mean[13] + mean[5] + mean[6] + mean[7]) / (3 * L ** 3))
        kts.append(mean[4])
    ps = np.array(ps)
    return ps.mean(), ps.std(ddof=1) / math.sqrt(blocks), float(np.mean(kts))


@pytest.mark.slow
@pytest.mark.parametrize("A,B,rho,L,sweeps,delta", [
    (25.0, 0.0, 3.0, 5.0, 300, 0.25),      # original DPD (Fig. 3a parameters)
    (-40.0, 25.0, 6.0, 4.0, 400, 0.12),    # mDPD (Fig. 3b parameters)
])
def test_pressure_matches_monte_carlo(A, B, rho, L, sweeps, delta):
    p_mc, e_mc, acc = mc_pressure(A, B, rho, L, sweeps=sweeps, burn=sweeps // 4,
                                  delta=delta, seed=1)
    assert 0.1 < acc < 0.9
    p_md, e_md, kT = _dpd_pressure(A, B, rho, L)
    assert abs(kT - 1.0) < 0.02
    assert abs(p_md - p_mc) < 4 * math.hypot(e_mc, e_md) + 0.1, (p_md, e_md, p_mc, e_mc)


@pytest.mark.slow
def test_eos_fits_of_fig3(golden_dir):
    """Fig. 3: the DPD quadratic EOS (a = 25) and the mDPD EOS (A = -40, B = 25),
    both fits, within their quality: 10% of the excess pressure for (a), and
    +-2.5 pressure units around rho = 6 for (b), where p crosses zero
    (coexistence near rho = 6.1)."""
    g = _golden(golden_dir)
    a = g["dpd_a"]
    p, e, _ = _dpd_pressure(a, 0.0, 3.0, 5.0, blocks=5)
    fit = 3.0 + g["dpd_coef"] * a * 9.0
    assert abs((p - 3.0) - (fit - 3.0)) < 0.1 * (fit - 3.0)
    A, B, rd, al, c, d = (g[k] for k in ("mdpd_A", "mdpd_B", "mdpd_rd", "mdpd_alpha",
                                         "mdpd_c", "mdpd_d"))
    rho = 6.0
    fit = rho + al * A * rho ** 2 + 2 * al * B * rd ** 4 * (rho ** 3 - c * rho ** 2 + d)
    p, e, _ = _dpd_pressure(A, B, rho, 5.0, blocks=5)
    assert abs(p - fit) < 2.5, (p, fit)


def _eos_zero(g):
    """Zero of the Fig. 3b mDPD EOS (alpha reading) near rho = 6, by bisection."""
    A, B, rd, al, c, d = (g[k] for k in ("mdpd_A", "mdpd_B", "mdpd_rd", "mdpd_alpha",
                                         "mdpd_c", "mdpd_d"))

    def p(rho):
        return rho + al * A * rho ** 2 + 2 * al * B * rd ** 4 * (rho ** 3 - c * rho ** 2 + d)
    lo, hi = 5.0, 8.0
    assert p(lo) < 0 < p(hi)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if p(mid) < 0 else (lo, mid)
    return 0.5 * (lo + hi)


@pytest.mark.slow
def test_slab_liquid_density_is_eos_coexistence(golden_dir):
    """A liquid slab in vacuum (Sec. 4.1 set-up with the Fig. 3b parameters)
    relaxes to zero pressure, so its interior density is the zero of the
    printed mDPD equation of state (6.10)."""
    rho0 = _eos_zero(_golden(golden_dir))
    assert abs(rho0 - 6.10) < 0.01
    Lx = 24.0
    w = I.slab(box=(Lx, 8.0, 8.0), slab_x=(8.0, 16.0), seed=7, precision=0, fill="lattice")
    o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed, use_cells=True)
    o.run(600)
    prof = []
    for _ in range(12):
        o.run(50)
        x = o.x[:, 0]
        th = 2 * np.pi * x / Lx
        com = Lx / (2 * np.pi) * np.arctan2(np.sin(th).mean(), np.cos(th).mean())
        h, _ = np.histogram((x - com + Lx / 2) % Lx, bins=12, range=(0, Lx))
        prof.append(h / (2.0 * 64.0))
    centre = np.mean(prof, axis=0)[4:8].mean()
    assert abs(centre - rho0) < 0.15, centre
