"""Pins of the oracle's wall-particle density phi (Sec. 3.2, Algorithm 1):
phi_i = sum over frozen j with 0 < r_ij < r_c of 15/(2 pi r_c^3)(1 - r/r_c)^2,
for mobile i; 0 for frozen i.

The pins do not restate the weight: a hand case with a literal value, and the
continuum limit of a flat wall, where a fine lattice of wall particles of
number density rho_w, filling the half-space z < 0, gives at height h above it
    phi(h) / rho_w = int_{z < 0, r < r_c} w(r) dV
                   = (2 - 5 t + 10 t^3 - 10 t^4 + 3 t^5) / 4,   t = h / r_c,
(the spherical-cap area 2 pi r (r - h) times the weight, integrated over r from
h to r_c); at the wall phi = rho_w / 2 because the weight integrates to one.
"""
import numpy as np

from oracle import oracle as O
from paper_1903_10134_gb300 import inputs as I


def _params(L, rc=1.0, rd=0.75, periodic=(1, 1, 0), lo=(0.0, 0.0, -1.5), hz=3.2):
    p = I.MDPDParams(box_lo=lo, box=(L, L, hz), periodic=periodic, ntypes=2, frozen_types=(1,))
    p.rc, p.rd = rc, rd
    return p


def test_wall_density_hand_case():
    """Probe at the origin; frozen particles at r = r_c/2 (weight
    15/(8 pi r_c^3) = 0.5968310365946075 for r_c = 1), at r = 1.2 r_c
    (outside), and a mobile particle at r = 0.3 (not counted).  Frozen
    particles get 0 whatever their neighbours."""
    p = _params(6.0, periodic=(0, 0, 0), lo=(-3.0, -3.0, -3.0), hz=6.0)
    x = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.0, 0.0, -1.2], [0.0, 0.3, 0.0],
                  [0.0, 0.5, 0.0]])
    typ = np.array([0, 1, 1, 0, 1], np.int32)
    for cells in (False, True):
        o = O.Oracle(p, x, np.zeros_like(x), typ, 1, use_cells=cells)
        phi = o.wall_density()
        assert abs(phi[0] - 2 * 0.5968310365946075) < 1e-15
        assert phi[1] == 0.0 and phi[2] == 0.0 and phi[4] == 0.0
        # the mobile particle at (0, 0.3, 0): frozen ones at distances
        # sqrt(0.34), 0.2 and sqrt(1.53) (outside)
        w = lambda r: 15 / (2 * np.pi) * (1 - r) ** 2   # noqa: E731  (r_c = 1)
        assert abs(phi[3] - (w(np.sqrt(0.34)) + w(0.2))) < 1e-14


def test_wall_density_flat_wall_closed_form():
    """Simple-cubic lattice (spacing a = 0.1 r_c) filling z < 0, probes at
    heights h over random lateral positions; the lattice sum approaches the
    continuum closed form at O(a^2): 1.5e-3 of rho_w at a = 0.1."""
    a, L = 0.1, 3.0
    m, nz = int(round(L / a)), int(round(1.2 / a))
    g = np.arange(m) * a + a / 2
    X, Y, Z = np.meshgrid(g, g, -(np.arange(nz) + 0.5) * a, indexing="ij")
    wall = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    hs = np.array([0.0, 0.1, 0.25, 0.4, 0.6, 0.8, 0.95, 1.05])
    rng = np.random.default_rng(0)
    probes = np.array([[rng.uniform(0, L), rng.uniform(0, L), h] for h in hs for _ in range(6)])
    x = np.concatenate([probes, wall])
    typ = np.concatenate([np.zeros(len(probes), np.int32), np.ones(len(wall), np.int32)])
    o = O.Oracle(_params(L), x, np.zeros_like(x), typ, 1, use_cells=True)
    phi = o.wall_density()
    got = phi[:len(probes)].reshape(len(hs), 6) * a ** 3
    t = np.minimum(hs, 1.0)
    want = (2 - 5 * t + 10 * t ** 3 - 10 * t ** 4 + 3 * t ** 5) / 4
    assert np.abs(got - want[:, None]).max() < 1.5e-3, (got.mean(1), want)
    assert np.all(phi[len(probes):] == 0.0)
    # at the wall: half the wall density
    assert abs(got[0].mean() - 0.5) < 1e-3
