"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
import this module.  It loads ``libmdpd_oracle.so`` (built from
``mdpd_oracle.c`` by ``oracle/build.py``) and shares nothing with the CUDA
library.  Parameters arrive as any object with the attributes of
``MDPDParams`` (box_lo, box, periodic, rc, rd, dt, kT, ntypes, A, B, gamma, g,
frozen_mask, xi_dist, rho_self).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MAXT = 8
_lib = None


class OrcSys(C.Structure):
    _fields_ = [
        ("lo", C.c_double * 3),
        ("L", C.c_double * 3),
        ("periodic", C.c_int32 * 3),
        ("ntypes", C.c_int32),
        ("rc", C.c_double), ("rd", C.c_double), ("dt", C.c_double), ("kT", C.c_double),
        ("A", (C.c_double * MAXT) * MAXT),
        ("B", (C.c_double * MAXT) * MAXT),
        ("gamma", (C.c_double * MAXT) * MAXT),
        ("g", C.c_double * 3),
        ("frozen_mask", C.c_uint32),
        ("xi_dist", C.c_int32),
        ("rho_self", C.c_int32),
        ("use_cells", C.c_int32),
        ("seed", C.c_uint64),
        ("mask", C.c_void_p),
        ("mdim", C.c_int32 * 3),
        ("pad_", C.c_int32),
        ("voxel", C.c_double),
        ("morigin", C.c_double * 3),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        d, i64, u64, i32, u32 = C.c_double, C.c_int64, C.c_uint64, C.c_int32, C.c_uint32
        P = C.c_void_p
        _lib.orc_philox4x32_10.argtypes = [P, P, P]
        _lib.orc_xi.argtypes = [u64, u64, u32, u32, i32]
        _lib.orc_xi.restype = d
        _lib.orc_w_rho.argtypes = [d, d]
        _lib.orc_w_rho.restype = d
        _lib.orc_pair_force.argtypes = [P, P, P, i32, i32, d, d, d, P, P]
        _lib.orc_pair_force.restype = C.c_int
        _lib.orc_density.argtypes = [P, i64, P, P]
        _lib.orc_wall_density.argtypes = [P, i64, P, P, P]
        _lib.orc_forces.argtypes = [P, i64, P, P, P, P, P, u64, P, P]
        _lib.orc_blocked.argtypes = [P, P]
        _lib.orc_observables.argtypes = [P, i64, P, P, P, u64, P]
        _lib.orc_observables.restype = None
        _lib.orc_run.argtypes = [P, i64, P, P, P, P, P, P, P, i64, P, P]
        _lib.orc_place_walls.argtypes = [P, P, P, d, P, d, d, u64, P, i64, P]
        _lib.orc_place_walls.restype = i64
        _lib.orc_num_threads.restype = C.c_int
        _lib.orc_set_num_threads.argtypes = [C.c_int]
        _lib.orc_set_num_threads.restype = None
        _lib.orc_forces_subset.argtypes = [P, i64, P, P, P, P, P, u64, i64, P, P]
        _lib.orc_force_vjp.argtypes = [P, i64, P, P, P, P, u64, P, P, P, P]
        _lib.orc_eval_vjp.argtypes = [P, i64, P, P, P, P, u64, P, P, P, P, P, P]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def make_sys(params, seed: int = 1, use_cells: bool = False, mask=None,
             voxel: float = 0.0, origin=(0.0, 0.0, 0.0)) -> tuple[OrcSys, object]:
    """Fill the oracle's parameter struct.  mask is indexed [z, y, x]."""
    s = OrcSys()
    for k in range(3):
        s.lo[k] = float(params.box_lo[k])
        s.L[k] = float(params.box[k])
        s.periodic[k] = int(params.periodic[k])
        s.g[k] = float(params.g[k])
        s.morigin[k] = float(origin[k])
    s.ntypes = int(params.ntypes)
    s.rc, s.rd, s.dt, s.kT = float(params.rc), float(params.rd), float(params.dt), float(params.kT)
    for a in range(MAXT):
        for b in range(MAXT):
            s.A[a][b] = float(params.A[a][b])
            s.B[a][b] = float(params.B[a][b])
            s.gamma[a][b] = float(params.gamma[a][b])
    s.frozen_mask = int(params.frozen_mask)
    s.xi_dist = int(params.xi_dist)
    s.rho_self = int(params.rho_self)
    s.use_cells = 1 if use_cells else 0
    s.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    keep = None
    if mask is not None:
        keep = _c(mask, np.uint8)
        s.mask = keep.ctypes.data
        nz, ny, nx = keep.shape
        s.mdim[0], s.mdim[1], s.mdim[2] = nx, ny, nz
        s.voxel = float(voxel)
    return s, keep


def philox4x32_10(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def xi(seed: int, step: int, i: int, j: int, dist: int = 0) -> float:
    return lib().orc_xi(seed, step, i, j, dist)


def w_rho(r: float, rd: float) -> float:
    return lib().orc_w_rho(r, rd)


def pair_force(params, d, vij, ti, tj, rho_i, rho_j, xi_val):
    """Force on i from j for one pair (or None outside 0 < r < r_c), and the
    conservative virial terms."""
    s, _ = make_sys(params)
    d = _c(d, np.float64)
    v = _c(vij, np.float64)
    f = np.zeros(3)
    w = np.zeros(6)
    ok = lib().orc_pair_force(C.byref(s), _ptr(d), _ptr(v), int(ti), int(tj),
                              float(rho_i), float(rho_j), float(xi_val), _ptr(f), _ptr(w))
    return (f, w) if ok else (None, None)


def place_walls(mask, periodic, voxel: float, origin, rho_w: float, shell: float,
                seed: int):
    """Wall-particle packing of a [z, y, x] solid mask; returns (positions,
    shell voxels as a [z, y, x] uint8 array)."""
    m = _c(mask, np.uint8)
    nz, ny, nx = m.shape
    dim = np.array([nx, ny, nz], np.int32)
    per = np.array([int(x) for x in periodic], np.int32)
    org = _c(origin, np.float64)
    shell_out = np.zeros_like(m)
    n = lib().orc_place_walls(_ptr(m), _ptr(dim), _ptr(per), float(voxel), _ptr(org),
                              float(rho_w), float(shell), int(seed), None, 0, _ptr(shell_out))
    out = np.zeros((max(n, 1), 3))
    n2 = lib().orc_place_walls(_ptr(m), _ptr(dim), _ptr(per), float(voxel), _ptr(org),
                               float(rho_w), float(shell), int(seed), _ptr(out), n, None)
    assert n2 == n
    return out[:n], shell_out


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of later oracle calls (results do not depend on it)."""
    lib().orc_set_num_threads(int(n))


class Oracle:
    """A whole mDPD system advanced by the oracle in FP64.

    State (pos, vel, acc, rho) is kept in input order with ids 0..n-1.  On
    construction the density and the forces of the initial state are
    evaluated with step index `step` (0 by default, as the library does at
    creation).
    """

    def __init__(self, params, pos, vel, type, seed: int, mask=None, voxel=0.0,
                 origin=(0.0, 0.0, 0.0), use_cells=None, ids=None, step: int = 0):
        self.params = params
        self.x = _c(pos, np.float64).copy()
        self.v = _c(vel, np.float64).copy()
        self.type = _c(type, np.int32).copy()
        n = self.x.shape[0]
        self.ids = _c(np.arange(n) if ids is None else ids, np.uint32).copy()
        if use_cells is None:
            use_cells = n > 2000 and all(
                (not params.periodic[k]) or params.box[k] >= 3 * params.rc for k in range(3))
        self.sys, self._mask = make_sys(params, seed, use_cells, mask, voxel, origin)
        self.a = np.zeros_like(self.x)
        self.rho = np.zeros(n)
        self.step = int(step)
        self.virial = np.zeros(6)
        self.refresh()

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def density(self, x=None) -> np.ndarray:
        x = self.x if x is None else _c(x, np.float64)
        rho = np.zeros(x.shape[0])
        if lib().orc_density(C.byref(self.sys), x.shape[0], _ptr(x), _ptr(rho)) != 0:
            raise RuntimeError("oracle density failed")
        return rho

    def wall_density(self, x=None) -> np.ndarray:
        """phi_i: density of frozen particles within r_c of each mobile particle,
        weight 15/(2 pi r_c^3)(1 - r/r_c)^2 (Sec. 3.2, Algorithm 1); 0 for
        frozen particles."""
        x = self.x if x is None else _c(x, np.float64)
        phi = np.zeros(x.shape[0])
        if lib().orc_wall_density(C.byref(self.sys), x.shape[0], _ptr(x), _ptr(self.type),
                                  _ptr(phi)) != 0:
            raise RuntimeError("oracle wall density failed")
        return phi

    def forces(self, x=None, v=None, rho=None, step=None):
        """Accelerations (m = 1, body force included, frozen = 0) and virial."""
        x = self.x if x is None else _c(x, np.float64)
        v = self.v if v is None else _c(v, np.float64)
        rho = self.density(x) if rho is None else _c(rho, np.float64)
        step = self.step if step is None else step
        a = np.zeros_like(x)
        vir = np.zeros(6)
        if lib().orc_forces(C.byref(self.sys), x.shape[0], _ptr(x), _ptr(v), _ptr(self.type),
                            _ptr(self.ids), _ptr(rho), int(step), _ptr(a), _ptr(vir)) != 0:
            raise RuntimeError("oracle forces failed")
        return a, vir

    def forces_subset(self, idx, x=None, v=None, rho=None, step=None):
        """Accelerations of the particles idx (rho of all particles needed)."""
        x = self.x if x is None else _c(x, np.float64)
        v = self.v if v is None else _c(v, np.float64)
        rho = self.density(x) if rho is None else _c(rho, np.float64)
        step = self.step if step is None else step
        idx = _c(idx, np.int64)
        a = np.zeros((idx.shape[0], 3))
        if lib().orc_forces_subset(C.byref(self.sys), x.shape[0], _ptr(x), _ptr(v),
                                   _ptr(self.type), _ptr(self.ids), _ptr(rho), int(step),
                                   idx.shape[0], _ptr(idx), _ptr(a)) != 0:
            raise RuntimeError("oracle forces failed")
        return a

    def force_vjp(self, abar, x=None, u=None, step=None):
        """(xbar, ubar, tbar) of L = sum_i abar_i . a_i(x, u, theta) at a fixed
        random stream; tbar[q][a][b] for q = A, B, gamma (symmetric entries)."""
        x = self.x if x is None else _c(x, np.float64)
        u = self.v if u is None else _c(u, np.float64)
        step = self.step if step is None else step
        ab = _c(abar, np.float64)
        xb = np.zeros_like(x)
        ub = np.zeros_like(x)
        tb = np.zeros((3, MAXT, MAXT))
        if lib().orc_force_vjp(C.byref(self.sys), x.shape[0], _ptr(x), _ptr(u), _ptr(self.type),
                               _ptr(self.ids), int(step), _ptr(ab), _ptr(xb), _ptr(ub),
                               _ptr(tb)) != 0:
            raise RuntimeError("oracle vjp failed")
        return xb, ub, tb

    def eval_vjp(self, abar=None, cvir=None, rhobar=None, x=None, u=None, step=None):
        """(xbar, ubar, tbar) of L = sum_i abar_i . a_i + sum_k cvir_k W_k +
        sum_i rhobar_i rho_i (accelerations, conservative virial in the order
        xx yy zz xy xz yz, local densities) at a fixed random stream; any of
        the three cotangents may be None."""
        x = self.x if x is None else _c(x, np.float64)
        u = self.v if u is None else _c(u, np.float64)
        step = self.step if step is None else step
        ab = None if abar is None else _c(abar, np.float64)
        cv = None if cvir is None else _c(cvir, np.float64)
        rb = None if rhobar is None else _c(rhobar, np.float64)
        xb = np.zeros_like(x)
        ub = np.zeros_like(x)
        tb = np.zeros((3, MAXT, MAXT))
        if lib().orc_eval_vjp(C.byref(self.sys), x.shape[0], _ptr(x), _ptr(u), _ptr(self.type),
                              _ptr(self.ids), int(step), None if ab is None else _ptr(ab),
                              None if cv is None else _ptr(cv), None if rb is None else _ptr(rb),
                              _ptr(xb), _ptr(ub), _ptr(tb)) != 0:
            raise RuntimeError("oracle vjp failed")
        return xb, ub, tb

    def refresh(self):
        """Recompute rho and a(t) of the current state (step index unchanged)."""
        self.rho = self.density()
        self.a, self.virial = self.forces(rho=self.rho)

    def run(self, nsteps: int):
        """Advance nsteps velocity-Verlet steps; returns (obs_last, obs_mean)."""
        step = C.c_uint64(self.step)
        last = np.zeros(16)
        s = np.zeros(16)
        rc = lib().orc_run(C.byref(self.sys), self.n, _ptr(self.x), _ptr(self.v),
                           _ptr(self.type), _ptr(self.ids), _ptr(self.a), _ptr(self.rho),
                           C.byref(step), int(nsteps), _ptr(last), _ptr(s))
        if rc != 0:
            raise RuntimeError("oracle run failed")
        self.step = int(step.value)
        if nsteps > 0:
            self.virial = last[5:11].copy()
        return last, s / max(nsteps, 1)

    def observables(self) -> np.ndarray:
        out = np.zeros(16)
        lib().orc_observables(C.byref(self.sys), self.n, _ptr(self.v), _ptr(self.type),
                              _ptr(self.virial), int(self.step), _ptr(out))
        return out

    def blocked(self, xn) -> bool:
        xn = _c(xn, np.float64)
        return bool(lib().orc_blocked(C.byref(self.sys), _ptr(xn)))
