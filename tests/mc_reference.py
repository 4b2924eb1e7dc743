"""Metropolis Monte Carlo of the mDPD potential: an equilibrium reference that
shares nothing with the oracle's dynamics.

The mDPD conservative force of Eq. 1 (arXiv:1903.10134) is the negative
gradient of
    U = sum_{i<j} (A r_c / 2)(1 - r_ij/r_c)^2  +  sum_i (pi r_d^4 B / 30) rho_i^2
with rho_i = sum_{j != i} 15/(2 pi r_d^3)(1 - r_ij/r_d)^2: differentiating the
second sum gives B (rho_i + rho_j)(1 - r/r_d) along r_ij.  A thermostat that
obeys the fluctuation-dissipation theorem (Sec. 2.1) samples exp(-U/kT), so
the time-averaged virial pressure of the dynamics must equal the Monte Carlo
average of the same virial in that ensemble.  Single-type, periodic cube.
"""
import math

import numpy as np


def _img(d, L):
    return d - L * np.round(d / L)


def mc_pressure(A, B, rho, L, rc=1.0, rd=0.75, kT=1.0, sweeps=600, burn=150,
                seed=0, delta=0.2, every=2):
    """Returns (mean pressure, standard error from 10 block means, acceptance)."""
    rng = np.random.default_rng(seed)
    N = int(round(rho * L ** 3))
    V = L ** 3
    x = rng.random((N, 3)) * L
    cw = 15.0 / (2 * math.pi * rd ** 3)
    cB = math.pi * rd ** 4 * B / 30.0

    def w_rho(r):
        return np.where(r < rd, cw * (1 - r / rd) ** 2, 0.0)

    def u_a(r):
        return np.where(r < rc, 0.5 * A * rc * (1 - r / rc) ** 2, 0.0)

    # initial local densities
    d = _img(x[:, None, :] - x[None, :, :], L)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, 10 * L)
    rhob = w_rho(r).sum(axis=1)

    samples = []
    acc = 0
    idx = np.arange(N)
    for sweep in range(sweeps):
        for i in rng.permutation(N):
            mask = idx != i
            xo = x[mask]
            ro = np.sqrt((_img(x[i] - xo, L) ** 2).sum(1))
            xn = (x[i] + delta * (2 * rng.random(3) - 1)) % L
            rn = np.sqrt((_img(xn - xo, L) ** 2).sum(1))
            wo, wn = w_rho(ro), w_rho(rn)
            rho_j_old = rhob[mask]
            rho_j_new = rho_j_old - wo + wn
            rho_i_new = wn.sum()
            dU = (u_a(rn) - u_a(ro)).sum()
            dU += cB * ((rho_j_new ** 2 - rho_j_old ** 2).sum() + rho_i_new ** 2 - rhob[i] ** 2)
            if dU <= 0 or rng.random() < math.exp(-dU / kT):
                x[i] = xn
                rhob[mask] = rho_j_new
                rhob[i] = rho_i_new
                acc += 1
        if sweep >= burn and (sweep - burn) % every == 0:
            d = _img(x[:, None, :] - x[None, :, :], L)
            r = np.sqrt((d * d).sum(-1))
            iu = np.triu_indices(N, 1)
            rr = r[iu]
            m = rr < rc
            rr = rr[m]
            ri = rhob[iu[0]][m]
            rj = rhob[iu[1]][m]
            fc = A * (1 - rr / rc) + np.where(rr < rd, B * (ri + rj) * (1 - rr / rd), 0.0)
            samples.append(N * kT / V + (fc * rr).sum() / (3 * V))
    s = np.array(samples)
    blocks = np.array_split(s, 10)
    bm = np.array([b.mean() for b in blocks])
    return s.mean(), bm.std(ddof=1) / math.sqrt(len(bm)), acc / (sweeps * N)
