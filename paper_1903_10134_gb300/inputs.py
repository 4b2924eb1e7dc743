"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds parameters and input generators only -- none of the mDPD
arithmetic (densities, forces, integration, wall packing) lives here.  The
workloads are shaped like the paper's (arXiv:1903.10134): the 10^3 periodic
bulk box of the EOS check (Fig. 3), a liquid slab (Sec. 4.1), a slit pore
(Sec. 4.2) and a voxelised porous rock (Sec. 5-6).  The paper's FIB-SEM images
are not available; a thresholded Gaussian random field stands in for them.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

MAX_TYPES = 8


def _table(value: float) -> np.ndarray:
    return np.full((MAX_TYPES, MAX_TYPES), float(value), dtype=np.float64)


@dataclass
class MDPDParams:
    """Physical and numerical parameters of one mDPD system (DPD units, m = 1)."""

    box_lo: tuple = (0.0, 0.0, 0.0)
    box: tuple = (10.0, 10.0, 10.0)
    periodic: tuple = (1, 1, 1)
    rc: float = 1.0
    rd: float = 0.75
    dt: float = 0.01
    kT: float = 1.0
    ntypes: int = 1
    A: np.ndarray = field(default_factory=lambda: _table(-40.0))
    B: np.ndarray = field(default_factory=lambda: _table(25.0))
    gamma: np.ndarray = field(default_factory=lambda: _table(4.5))
    g: tuple = (0.0, 0.0, 0.0)
    frozen_types: tuple = ()
    precision: int = 1          # 0 = FP64 pair arithmetic, 1 = FP32
    xi_dist: int = 0            # 0 = uniform unit variance, 1 = Gaussian
    rho_self: int = 0

    @property
    def frozen_mask(self) -> int:
        m = 0
        for t in self.frozen_types:
            m |= 1 << int(t)
        return m

    def set_pair(self, ti: int, tj: int, A=None, B=None, gamma=None) -> "MDPDParams":
        for name, val in (("A", A), ("B", B), ("gamma", gamma)):
            if val is not None:
                tab = getattr(self, name)
                tab[ti, tj] = val
                tab[tj, ti] = val
        return self

    def copy(self, **kw) -> "MDPDParams":
        p = dataclasses.replace(self, A=self.A.copy(), B=self.B.copy(),
                                gamma=self.gamma.copy())
        for k, v in kw.items():
            setattr(p, k, v)
        return p


@dataclass
class Workload:
    """A system ready to hand to either implementation."""

    name: str
    params: MDPDParams
    pos: np.ndarray            # (n, 3) float64
    vel: np.ndarray            # (n, 3) float64
    type: np.ndarray           # (n,) int32
    seed: int
    mask: np.ndarray | None = None       # (nz, ny, nx) uint8 solid voxels, or None
    voxel: float = 0.0
    origin: tuple = (0.0, 0.0, 0.0)
    wall_density: float = 0.0
    shell: float = 0.0
    wall_type: int = 1
    wall_seed: int = 0
    steps: int = 0

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def maxwell_velocities(n: int, kT: float, rng: np.random.Generator) -> np.ndarray:
    """Maxwell-Boltzmann velocities at temperature kT (m = 1), zero total momentum."""
    v = rng.normal(0.0, np.sqrt(kT), size=(n, 3))
    if n > 1:
        v -= v.mean(axis=0, keepdims=True)
    return v


def uniform_positions(n: int, lo, hi, rng: np.random.Generator) -> np.ndarray:
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lo + (hi - lo) * rng.random((n, 3))


def bulk(n: int = 6000, L=(10.0, 10.0, 10.0), seed: int = 1, precision: int = 0,
         steps: int = 100, **pk) -> Workload:
    """Periodic bulk liquid: the 10^3 box of the EOS validation (Fig. 3b),
    uniform random positions, Maxwell velocities at kT = 1."""
    rng = np.random.default_rng(seed)
    p = MDPDParams(box=tuple(float(x) for x in L), precision=precision, **pk)
    pos = uniform_positions(n, p.box_lo, np.add(p.box_lo, p.box), rng)
    vel = maxwell_velocities(n, p.kT, rng)
    return Workload("bulk", p, pos, vel, np.zeros(n, np.int32), seed, steps=steps)


def lattice_positions(lo, hi, density: float, rng: np.random.Generator,
                      jitter: float = 0.05) -> np.ndarray:
    """Simple cubic lattice filling [lo, hi) at about the given number density
    (an integer number of sites per edge), each site displaced by up to
    `jitter` lattice spacings."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    a0 = density ** (-1.0 / 3.0)
    m = np.maximum(1, np.round((hi - lo) / a0)).astype(int)
    a = (hi - lo) / m
    g = np.stack(np.meshgrid(*[np.arange(k) for k in m], indexing="ij"), -1).reshape(-1, 3)
    pos = lo + (g + 0.5) * a
    return pos + jitter * a * (2 * rng.random(pos.shape) - 1)


def slab(box=(60.0, 20.0, 20.0), slab_x=(20.0, 40.0), density: float = 6.0,
         seed: int = 1, precision: int = 1, steps: int = 20000, fill: str = "random",
         **pk) -> Workload:
    """Liquid-vapour slab (Sec. 4.1 shape): a block of liquid across the full
    y-z section of a periodic box, vapour elsewhere.  fill = "random" places
    the particles uniformly at random, "lattice" on a jittered cubic lattice
    (the paper starts its slab from an fcc lattice)."""
    rng = np.random.default_rng(seed)
    p = MDPDParams(box=tuple(float(x) for x in box), precision=precision, **pk)
    lo, hi = (slab_x[0], 0.0, 0.0), (slab_x[1], box[1], box[2])
    if fill == "lattice":
        pos = lattice_positions(lo, hi, density, rng)
    else:
        vol = (slab_x[1] - slab_x[0]) * box[1] * box[2]
        pos = uniform_positions(int(round(density * vol)), lo, hi, rng)
    n = pos.shape[0]
    vel = maxwell_velocities(n, p.kT, rng)
    return Workload("slab", p, pos, vel, np.zeros(n, np.int32), seed, steps=steps)


def _fluid_in_pores(mask: np.ndarray, voxel: float, origin, density: float,
                    rng: np.random.Generator) -> np.ndarray:
    """Uniform random fluid positions at the given number density inside the
    pore (mask == 0) voxels.  mask is indexed [z, y, x]."""
    pore = np.flatnonzero(mask.reshape(-1) == 0)
    nz, ny, nx = mask.shape
    n = int(round(density * pore.size * voxel ** 3))
    pick = pore[rng.integers(0, pore.size, size=n)]
    ix = pick % nx
    iy = (pick // nx) % ny
    iz = pick // (nx * ny)
    idx = np.stack([ix, iy, iz], axis=1).astype(np.float64)
    return np.asarray(origin, np.float64) + (idx + rng.random((n, 3))) * voxel


def slit(Lx: float = 100.0, Ly: float = 40.0, H: float = 20.0, wall: float = 1.0,
         voxel: float = 0.5, density: float = 6.0, A_fs: float = -30.0,
         g: float = 0.02, seed: int = 1, precision: int = 1,
         steps: int = 50000) -> Workload:
    """Slit pore (Sec. 4.2 / Poiseuille shape): periodic in x and y, fluid in
    0 <= z < H, solid slabs of thickness `wall` on both sides given as a voxel
    mask; the wall particles come from the library's wall packing."""
    rng = np.random.default_rng(seed)
    lo = (0.0, 0.0, -wall)
    box = (Lx, Ly, H + 2 * wall)
    p = MDPDParams(box_lo=lo, box=box, periodic=(1, 1, 0), ntypes=2,
                   g=(g, 0.0, 0.0), frozen_types=(1,), precision=precision)
    p.set_pair(0, 1, A=A_fs)
    nx, ny, nz = (int(round(b / voxel)) for b in box)
    zc = lo[2] + (np.arange(nz) + 0.5) * voxel
    solid_z = (zc < 0.0) | (zc >= H)
    mask = np.broadcast_to(solid_z[:, None, None], (nz, ny, nx)).astype(np.uint8).copy()
    pos = _fluid_in_pores(mask, voxel, lo, density, rng)
    vel = maxwell_velocities(pos.shape[0], p.kT, rng)
    return Workload("slit", p, pos, vel, np.zeros(pos.shape[0], np.int32), seed,
                    mask=mask, voxel=voxel, origin=lo, wall_density=density,
                    shell=wall, wall_type=1, wall_seed=seed + 1000, steps=steps)


def gaussian_random_field(n, corr: float, rng: np.random.Generator) -> np.ndarray:
    """Periodic Gaussian random field on an n^3 (or (nz, ny, nx)) grid with
    covariance exp(-r^2 / (2 corr^2)) (r, corr in voxels), by filtering white
    noise in Fourier space with exp(-k^2 corr^2 / 4)."""
    shape = (n, n, n) if np.isscalar(n) else tuple(n)
    white = rng.standard_normal(shape)
    kz = np.fft.fftfreq(shape[0]) * 2 * np.pi
    ky = np.fft.fftfreq(shape[1]) * 2 * np.pi
    kx = np.fft.rfftfreq(shape[2]) * 2 * np.pi
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    spec = np.fft.rfftn(white) * np.exp(-k2 * corr * corr / 4.0)
    return np.fft.irfftn(spec, s=shape, axes=(0, 1, 2))


def rock(nvox: int = 256, voxel: float = 0.5, corr: float = 4.0,
         porosity: float = 0.15, density: float = 6.0, shell: float = 1.0,
         A_fs: float = -40.0, g: float = 0.01, seed: int = 1, precision: int = 1,
         steps: int = 10000) -> Workload:
    """Synthetic nanoporous rock: a periodic nvox^3 Gaussian random field
    (correlation length `corr` voxels) thresholded so that a fraction
    `porosity` of the voxels is pore; fluid at `density` in the pores; wall
    particles (from the library's packing) in a `shell`-thick solid layer."""
    rng = np.random.default_rng(seed)
    field_ = gaussian_random_field(nvox, corr, rng)
    thr = np.quantile(field_, porosity)
    mask = (field_ >= thr).astype(np.uint8)          # 1 = solid
    L = nvox * voxel
    p = MDPDParams(box=(L, L, L), periodic=(1, 1, 1), ntypes=2,
                   g=(g, 0.0, 0.0), frozen_types=(1,), precision=precision)
    p.set_pair(0, 1, A=A_fs)
    pos = _fluid_in_pores(mask, voxel, (0.0, 0.0, 0.0), density, rng)
    vel = maxwell_velocities(pos.shape[0], p.kT, rng)
    return Workload("rock", p, pos, vel, np.zeros(pos.shape[0], np.int32), seed,
                    mask=mask, voxel=voxel, origin=(0.0, 0.0, 0.0),
                    wall_density=density, shell=shell, wall_type=1,
                    wall_seed=seed + 1000, steps=steps)


def tiny(n: int, L, seed: int, periodic=(1, 1, 1), ntypes: int = 1,
         precision: int = 0, spread: float = 1.0, **pk) -> Workload:
    """A small random system for brute-force and parity checks; with ntypes > 1
    the types are drawn uniformly and the A/B/gamma tables get distinct
    seeded entries so that a transposed table lookup shows up."""
    rng = np.random.default_rng(seed)
    p = MDPDParams(box=tuple(float(x) for x in L), periodic=tuple(periodic),
                   ntypes=ntypes, precision=precision, **pk)
    if ntypes > 1:
        for ti in range(ntypes):
            for tj in range(ti, ntypes):
                p.set_pair(ti, tj, A=-50.0 + 20.0 * rng.random(),
                           B=15.0 + 20.0 * rng.random(),
                           gamma=3.0 + 3.0 * rng.random())
    pos = uniform_positions(n, p.box_lo, np.add(p.box_lo, p.box), rng)
    vel = spread * maxwell_velocities(n, p.kT, rng)
    typ = rng.integers(0, ntypes, size=n).astype(np.int32)
    return Workload("tiny", p, pos, vel, typ, seed)


def water_slab(seed: int = 1, precision: int = 1, steps: int = 10000) -> Workload:
    """Water liquid-vacuum slab of Sec. 4.1: periodic box [-50, 50]^3, an fcc
    slab with lattice constant r_c filling -10 <= x <= 10 (41 planes of 2 x 100
    x 100 sites: 820,000 particles), A = -50, B = 25, r_d = 0.75, gamma = 12.4,
    Maxwell velocities at kT = 1."""
    rng = np.random.default_rng(seed)
    p = MDPDParams(box_lo=(-50.0, -50.0, -50.0), box=(100.0, 100.0, 100.0),
                   precision=precision)
    p.A[:] = -50.0
    p.B[:] = 25.0
    p.gamma[:] = 12.4
    j, k = np.meshgrid(np.arange(100.0), np.arange(100.0), indexing="ij")
    j = j.ravel()
    k = k.ravel()
    planes = []
    for m in range(41):
        x = -10.0 + 0.5 * m
        if m % 2 == 0:
            yz = [(j, k), (j + 0.5, k + 0.5)]
        else:
            yz = [(j + 0.5, k), (j, k + 0.5)]
        for y, z in yz:
            planes.append(np.stack([np.full_like(y, x), y - 50.0, z - 50.0], 1))
    pos = np.concatenate(planes)
    vel = maxwell_velocities(pos.shape[0], p.kT, rng)
    return Workload("water_slab", p, pos, vel, np.zeros(pos.shape[0], np.int32), seed,
                    steps=steps)


def contact_slit(A_sl: float, seed: int = 1, precision: int = 1, steps: int = 14000) -> Workload:
    """Static contact angle set-up of Sec. 4.2: x in [-30, 30] and z in
    [-2.5, 2.5] periodic, walls for |y| > 4 (solid voxels of 0.5, wall particles
    at density 35/6 so that the two walls hold about 3,500), 4,000 liquid
    particles placed at random in -13 <= x <= 13, |y| <= 4, A_LL = -40,
    A_SL given, B = 25, r_d = 0.75."""
    rng = np.random.default_rng(seed)
    lo = (-30.0, -5.0, -2.5)
    box = (60.0, 10.0, 5.0)
    p = MDPDParams(box_lo=lo, box=box, periodic=(1, 0, 1), ntypes=2, frozen_types=(1,),
                   precision=precision)
    p.set_pair(0, 1, A=A_sl)
    voxel = 0.5
    nx, ny, nz = (int(round(b / voxel)) for b in box)
    yc = lo[1] + (np.arange(ny) + 0.5) * voxel
    solid_y = np.abs(yc) > 4.0
    mask = np.broadcast_to(solid_y[None, :, None], (nz, ny, nx)).astype(np.uint8).copy()
    pos = uniform_positions(4000, (-13.0, -4.0, -2.5), (13.0, 4.0, 2.5), rng)
    vel = maxwell_velocities(4000, p.kT, rng)
    return Workload("contact_slit", p, pos, vel, np.zeros(4000, np.int32), seed, mask=mask,
                    voxel=voxel, origin=lo, wall_density=35.0 / 6.0, shell=1.0, wall_type=1,
                    wall_seed=seed + 1000, steps=steps)


def batch_slabs(nrep: int = 256, n_range=(2000, 20000), A_range=(-50.0, -30.0),
                B_range=(15.0, 35.0), seed: int = 1, precision: int = 1,
                steps: int = 50, density: float = 6.0) -> list:
    """Many small liquid slabs of uneven size and parameters, advanced together
    as one batch (ensembles or A, B sweeps and fits).  Replica r: N_r drawn
    uniformly from n_range, A_r and B_r uniformly from their ranges, a periodic
    box 3 L x L x L with L = (N_r / density)^(1/3) holding a liquid block of
    density `density` over its middle third in x (random positions), Maxwell
    velocities at kT = 1, seed `seed` + r.  `steps` is the length of one
    window."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(nrep):
        n_r = int(rng.integers(n_range[0], n_range[1] + 1))
        A = float(rng.uniform(*A_range))
        B = float(rng.uniform(*B_range))
        L = (n_r / density) ** (1.0 / 3.0)
        p = MDPDParams(box=(3 * L, L, L), precision=precision)
        p.set_pair(0, 0, A=A, B=B)
        pos = uniform_positions(n_r, (L, 0.0, 0.0), (2 * L, L, L), rng)
        vel = maxwell_velocities(n_r, p.kT, rng)
        out.append(Workload("batch_slab", p, pos, vel, np.zeros(n_r, np.int32), seed + r,
                            steps=steps))
    return out
