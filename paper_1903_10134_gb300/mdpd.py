"""Thin ctypes binding of the C ABI in ``include/mdpd.h``.

Every function here only marshals arguments to the entry point of the same
name in ``libmdpd_gb300.so``; all of the method's work runs in the library's
sm_103a kernels.  Importing this module loads nothing; the first call loads
the library (building it if it is missing or stale) and raises if it cannot.
There is no CPU fallback.

Host arrays are numpy float64 (positions/velocities as (n, 3)), int32 types;
``*_dev`` variants take CUDA torch tensors of the same shapes and dtypes.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

MAX_TYPES = 8
NUM_OBS = 16
OPT_GRAPH = 1
OPT_PROFILE = 2
OPT_KERNELS = 3
OPT_PROFILE_EVERY = 4
OPT_WALL_DENSITY = 5
OPT_FORCE_LANES = 6
OPT_DENSITY_SHAPE = 7
KERNELS_NLIST = 0
KERNELS_SCAN = 1
KERNELS_NLIST_THREAD = 2
KCLASS = ("bin", "density", "force", "other")

ERRORS = {
    -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NONFINITE",
    -5: "OUT_OF_BOX", -6: "TILE_OVERFLOW", -7: "TIMEOUT", -8: "BOUNDS",
}

_lib = None


class MDPDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"MDPD_ERR_{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class Params(C.Structure):
    """Mirror of ``mdpd_params``."""

    _fields_ = [
        ("box_lo", C.c_double * 3),
        ("box", C.c_double * 3),
        ("periodic", C.c_int32 * 3),
        ("ntypes", C.c_int32),
        ("rc", C.c_double), ("rd", C.c_double), ("dt", C.c_double), ("kT", C.c_double),
        ("A", (C.c_double * MAX_TYPES) * MAX_TYPES),
        ("B", (C.c_double * MAX_TYPES) * MAX_TYPES),
        ("gamma", (C.c_double * MAX_TYPES) * MAX_TYPES),
        ("g", C.c_double * 3),
        ("frozen_type_mask", C.c_uint32),
        ("precision", C.c_int32),
        ("xi_dist", C.c_int32),
        ("rho_self", C.c_int32),
    ]


def to_c_params(p) -> Params:
    """Fill ``mdpd_params`` from any object with MDPDParams' attributes."""
    c = Params()
    for k in range(3):
        c.box_lo[k] = float(p.box_lo[k])
        c.box[k] = float(p.box[k])
        c.periodic[k] = int(p.periodic[k])
        c.g[k] = float(p.g[k])
    c.ntypes = int(p.ntypes)
    c.rc, c.rd, c.dt, c.kT = float(p.rc), float(p.rd), float(p.dt), float(p.kT)
    for a in range(MAX_TYPES):
        for b in range(MAX_TYPES):
            c.A[a][b] = float(p.A[a][b])
            c.B[a][b] = float(p.B[a][b])
            c.gamma[a][b] = float(p.gamma[a][b])
    c.frozen_type_mask = int(p.frozen_mask)
    c.precision = int(p.precision)
    c.xi_dist = int(p.xi_dist)
    c.rho_self = int(p.rho_self)
    return c


SYMBOLS = (
    "mdpd_create", "mdpd_create_dev", "mdpd_set_walls", "mdpd_step", "mdpd_sync",
    "mdpd_num_particles", "mdpd_step_count", "mdpd_get_state", "mdpd_get_state_dev",
    "mdpd_set_state", "mdpd_set_state_dev", "mdpd_forces", "mdpd_forces_dev",
    "mdpd_observables", "mdpd_observables_mean", "mdpd_pair_count", "mdpd_set_option",
    "mdpd_profile",
    "mdpd_describe", "mdpd_autotune", "mdpd_set_params", "mdpd_set_step",
    "mdpd_get_accel_dev", "mdpd_force_vjp_dev", "mdpd_get_wall_density", "mdpd_density_noalloc", "mdpd_destroy",
    "mdpd_last_error", "mdpd_create_batch", "mdpd_num_replicas", "mdpd_batch_observables",
    "mdpd_batch_set_params", "mdpd_measure_fma_peak", "mdpd_density_vjp_dev",
    "mdpd_get_accel", "mdpd_set_state_accel", "mdpd_eval_vjp_dev", "mdpd_window_forward",
    "mdpd_window_vjp_dev",
)


def debug_build() -> bool:
    """Whether this process uses the index-checking debug build of the library
    (environment variable MDPD_DEBUG=1)."""
    return os.environ.get("MDPD_DEBUG", "0") == "1"


def library_path() -> str:
    return _build.LIB_DEBUG if debug_build() else _build.LIB


def lib(build_if_stale: bool = True):
    """Load the CUDA library (compiling it first if it is missing or stale);
    the debug build when MDPD_DEBUG=1."""
    global _lib
    if _lib is not None:
        return _lib
    dbg = debug_build()
    path = _build.build(debug=dbg) if build_if_stale else library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    L = C.CDLL(path)
    P, i64, i32, u64, d = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_double
    L.mdpd_create.argtypes = [P, i64, P, P, P, u64, P, C.POINTER(P)]
    L.mdpd_create_dev.argtypes = [P, i64, P, P, P, u64, P, C.POINTER(P)]
    L.mdpd_set_walls.argtypes = [P, P, i32, i32, i32, d, P, d, d, i32, u64]
    L.mdpd_step.argtypes = [P, i64]
    L.mdpd_sync.argtypes = [P]
    L.mdpd_num_particles.argtypes = [P, C.POINTER(i64)]
    L.mdpd_step_count.argtypes = [P, C.POINTER(i64)]
    L.mdpd_get_state.argtypes = [P, P, P, P, P]
    L.mdpd_get_state_dev.argtypes = [P, P, P, P, P]
    L.mdpd_set_state.argtypes = [P, P, P]
    L.mdpd_set_state_dev.argtypes = [P, P, P]
    L.mdpd_forces.argtypes = [P, P, P]
    L.mdpd_forces_dev.argtypes = [P, P, P]
    L.mdpd_observables.argtypes = [P, P]
    L.mdpd_observables_mean.argtypes = [P, P, i32]
    L.mdpd_pair_count.argtypes = [P, C.POINTER(i64)]
    L.mdpd_set_option.argtypes = [P, i32, i64]
    L.mdpd_profile.argtypes = [P, P, C.POINTER(i64), C.POINTER(i64)]
    L.mdpd_describe.argtypes = [P, P, C.POINTER(i32)]
    L.mdpd_density_noalloc.argtypes = [P, i64, P, P, P]
    L.mdpd_autotune.argtypes = [P, i32, P, P]
    L.mdpd_set_params.argtypes = [P, P]
    L.mdpd_get_wall_density.argtypes = [P, P]
    L.mdpd_set_step.argtypes = [P, i64]
    L.mdpd_get_accel_dev.argtypes = [P, P]
    L.mdpd_force_vjp_dev.argtypes = [P, P, P, P, P]
    L.mdpd_create_batch.argtypes = [i32, P, P, P, P, P, P, P, C.POINTER(P)]
    L.mdpd_num_replicas.argtypes = [P, C.POINTER(i32)]
    L.mdpd_batch_observables.argtypes = [P, P, i32, i32]
    L.mdpd_batch_set_params.argtypes = [P, P]
    L.mdpd_measure_fma_peak.argtypes = [C.POINTER(d), C.POINTER(d)]
    L.mdpd_density_vjp_dev.argtypes = [P, P, P]
    L.mdpd_get_accel.argtypes = [P, P]
    L.mdpd_set_state_accel.argtypes = [P, P, P, P]
    L.mdpd_eval_vjp_dev.argtypes = [P, P, P, P, P, P, P]
    L.mdpd_window_forward.argtypes = [P, i32]
    L.mdpd_window_vjp_dev.argtypes = [P, P, P, P, P, P, P, P]
    L.mdpd_destroy.argtypes = [P]
    L.mdpd_destroy.restype = None
    L.mdpd_last_error.argtypes = [P]
    L.mdpd_last_error.restype = C.c_char_p
    for name in SYMBOLS:
        if name not in ("mdpd_destroy", "mdpd_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc: int, h=None):
    if rc != 0:
        msg = lib().mdpd_last_error(h)
        raise MDPDError(rc, msg.decode() if msg else "")


def _arr(a, dtype, shape=None) -> np.ndarray:
    out = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None and out.shape != shape:
        out = out.reshape(shape)
    return out


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _tptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device variants take contiguous CUDA tensors")
    return C.c_void_p(t.data_ptr())


# ---- entry points (same names as the C ABI) ------------------------------------

def mdpd_create(params, pos, vel, type, seed: int, stream=None):
    n = int(np.asarray(pos).shape[0])
    pos = _arr(pos, np.float64, (n, 3))
    vel = _arr(vel, np.float64, (n, 3))
    typ = _arr(type, np.int32, (n,))
    cp = to_c_params(params)
    h = C.c_void_p()
    _check(lib().mdpd_create(C.byref(cp), n, _p(pos), _p(vel), _p(typ), int(seed),
                             _stream_ptr(stream), C.byref(h)))
    return h


def mdpd_create_dev(params, pos_t, vel_t, type_t, seed: int, stream=None):
    n = int(pos_t.shape[0])
    cp = to_c_params(params)
    h = C.c_void_p()
    _check(lib().mdpd_create_dev(C.byref(cp), n, _tptr(pos_t), _tptr(vel_t), _tptr(type_t),
                                 int(seed), _stream_ptr(stream), C.byref(h)))
    return h


def mdpd_create_batch(params_list, n_list, pos, vel, type, seeds, stream=None):
    """params_list[r], n_list[r], seeds[r] per replica; pos/vel (N, 3), type (N,)
    with replica 0's particles first."""
    nrep = len(params_list)
    ns = _arr([int(v) for v in n_list], np.int64, (nrep,))
    N = int(ns.sum())
    pos = _arr(pos, np.float64, (N, 3))
    vel = _arr(vel, np.float64, (N, 3))
    typ = _arr(type, np.int32, (N,))
    cps = (Params * nrep)(*[to_c_params(p) for p in params_list])
    sd = _arr([int(v) for v in seeds], np.uint64, (nrep,))
    h = C.c_void_p()
    _check(lib().mdpd_create_batch(nrep, cps, _p(ns), _p(pos), _p(vel), _p(typ), _p(sd),
                                   _stream_ptr(stream), C.byref(h)))
    return h


def mdpd_num_replicas(h) -> int:
    r = C.c_int32()
    _check(lib().mdpd_num_replicas(h, C.byref(r)), h)
    return int(r.value)


def mdpd_batch_observables(h, mean: bool = False, reset: bool = False) -> np.ndarray:
    out = np.zeros((mdpd_num_replicas(h), NUM_OBS))
    _check(lib().mdpd_batch_observables(h, _p(out), int(mean), int(reset)), h)
    return out


def mdpd_batch_set_params(h, params_list):
    cps = (Params * len(params_list))(*[to_c_params(p) for p in params_list])
    _check(lib().mdpd_batch_set_params(h, cps), h)


def mdpd_set_walls(h, solid, voxel: float, origin, wall_density: float, shell_thickness: float,
                   wall_type: int, seed: int):
    """solid: uint8 array indexed [z, y, x] (x fastest in memory)."""
    m = _arr(solid, np.uint8)
    nz, ny, nx = m.shape
    org = _arr(origin, np.float64, (3,))
    _check(lib().mdpd_set_walls(h, _p(m), nx, ny, nz, float(voxel), _p(org),
                                float(wall_density), float(shell_thickness), int(wall_type),
                                int(seed)), h)


def mdpd_step(h, nsteps: int):
    _check(lib().mdpd_step(h, int(nsteps)), h)


def mdpd_sync(h):
    _check(lib().mdpd_sync(h), h)


def mdpd_num_particles(h) -> int:
    n = C.c_int64()
    _check(lib().mdpd_num_particles(h, C.byref(n)), h)
    return int(n.value)


def mdpd_step_count(h) -> int:
    n = C.c_int64()
    _check(lib().mdpd_step_count(h, C.byref(n)), h)
    return int(n.value)


def mdpd_get_state(h, pos=None, vel=None, want_type=True, want_rho=True):
    """Returns (pos, vel, type, rho); pos/vel may be caller buffers (e.g. pinned
    host memory viewed as numpy), type/rho are skipped when not wanted."""
    n = mdpd_num_particles(h)
    pos = np.zeros((n, 3)) if pos is None else pos
    vel = np.zeros((n, 3)) if vel is None else vel
    typ = np.zeros(n, np.int32) if want_type else None
    rho = np.zeros(n) if want_rho else None
    for a in (pos, vel):
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == 3 * n
    _check(lib().mdpd_get_state(h, _p(pos), _p(vel), None if typ is None else _p(typ),
                                None if rho is None else _p(rho)), h)
    return pos, vel, typ, rho


def mdpd_get_state_dev(h, pos_t=None, vel_t=None, type_t=None, rho_t=None):
    _check(lib().mdpd_get_state_dev(h, _tptr(pos_t), _tptr(vel_t), _tptr(type_t), _tptr(rho_t)), h)


def mdpd_set_state(h, pos, vel):
    n = mdpd_num_particles(h)
    pos = _arr(pos, np.float64, (n, 3))
    vel = _arr(vel, np.float64, (n, 3))
    _check(lib().mdpd_set_state(h, _p(pos), _p(vel)), h)


def mdpd_set_state_dev(h, pos_t, vel_t):
    _check(lib().mdpd_set_state_dev(h, _tptr(pos_t), _tptr(vel_t)), h)


def mdpd_forces(h):
    n = mdpd_num_particles(h)
    f = np.zeros((n, 3))
    rho = np.zeros(n)
    _check(lib().mdpd_forces(h, _p(f), _p(rho)), h)
    return f, rho


def mdpd_forces_dev(h, force_t=None, rho_t=None):
    _check(lib().mdpd_forces_dev(h, _tptr(force_t), _tptr(rho_t)), h)


def mdpd_observables(h) -> np.ndarray:
    out = np.zeros(NUM_OBS)
    _check(lib().mdpd_observables(h, _p(out)), h)
    return out


def mdpd_observables_mean(h, reset: bool = True) -> np.ndarray:
    out = np.zeros(NUM_OBS)
    _check(lib().mdpd_observables_mean(h, _p(out), 1 if reset else 0), h)
    return out


def mdpd_pair_count(h) -> int:
    n = C.c_int64()
    _check(lib().mdpd_pair_count(h, C.byref(n)), h)
    return int(n.value)


def mdpd_set_option(h, option: int, value: int):
    _check(lib().mdpd_set_option(h, int(option), int(value)), h)


def mdpd_profile(h):
    """Kernel time per class (ms, summed over recorded steps), steps, launches."""
    ms = np.zeros(len(KCLASS))
    steps = C.c_int64()
    launches = C.c_int64()
    _check(lib().mdpd_profile(h, _p(ms), C.byref(steps), C.byref(launches)), h)
    return dict(zip(KCLASS, ms.tolist())), int(steps.value), int(launches.value)


def mdpd_describe(h):
    nc = np.zeros(3, np.int32)
    lps = C.c_int32()
    _check(lib().mdpd_describe(h, _p(nc), C.byref(lps)), h)
    return nc.tolist(), int(lps.value)


def mdpd_get_accel(h, out=None) -> np.ndarray:
    """Accelerations the next half-kick uses (n, 3), into `out` if given (a
    C-contiguous float64 buffer, e.g. pinned host memory viewed as numpy)."""
    n = mdpd_num_particles(h)
    a = np.zeros((n, 3)) if out is None else out
    assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == 3 * n
    _check(lib().mdpd_get_accel(h, _p(a)), h)
    return a


def mdpd_set_state_accel(h, pos, vel, accel):
    n = mdpd_num_particles(h)
    pos = _arr(pos, np.float64, (n, 3))
    vel = _arr(vel, np.float64, (n, 3))
    acc = _arr(accel, np.float64, (n, 3))
    _check(lib().mdpd_set_state_accel(h, _p(pos), _p(vel), _p(acc)), h)


def mdpd_density_vjp_dev(h, rhobar_t, xbar_t):
    _check(lib().mdpd_density_vjp_dev(h, _tptr(rhobar_t), _tptr(xbar_t)), h)


def mdpd_get_wall_density(h) -> np.ndarray:
    phi = np.zeros(mdpd_num_particles(h))
    _check(lib().mdpd_get_wall_density(h, _p(phi)), h)
    return phi


def mdpd_set_params(h, params):
    cp = to_c_params(params)
    _check(lib().mdpd_set_params(h, C.byref(cp)), h)


def mdpd_set_step(h, step: int):
    _check(lib().mdpd_set_step(h, int(step)), h)


def mdpd_get_accel_dev(h, accel_t):
    _check(lib().mdpd_get_accel_dev(h, _tptr(accel_t)), h)


def mdpd_force_vjp_dev(h, abar_t, xbar_t=None, ubar_t=None, theta_bar_t=None):
    """VJP of one force evaluation at the current state (device tensors:
    abar/xbar/ubar (n, 3) float64, theta_bar (3, 8, 8) float64)."""
    _check(lib().mdpd_force_vjp_dev(h, _tptr(abar_t), _tptr(xbar_t), _tptr(ubar_t),
                                    _tptr(theta_bar_t)), h)


def mdpd_eval_vjp_dev(h, abar_t=None, cvir_t=None, rhobar_t=None, xbar_t=None, ubar_t=None,
                      theta_bar_t=None):
    """VJP of one evaluation (accelerations, virial, densities) at the current
    state; device tensors: abar/xbar/ubar (n, 3), cvir (nrep, 6), rhobar (n,),
    theta_bar (nrep, 3, 8, 8) (or (3, 8, 8) for a single system), float64."""
    _check(lib().mdpd_eval_vjp_dev(h, _tptr(abar_t), _tptr(cvir_t), _tptr(rhobar_t),
                                   _tptr(xbar_t), _tptr(ubar_t), _tptr(theta_bar_t)), h)


def mdpd_window_forward(h, nsteps: int):
    _check(lib().mdpd_window_forward(h, int(nsteps)), h)


def mdpd_window_vjp_dev(h, xbar_t=None, vbar_t=None, cvir_t=None, rhobar_t=None, x0bar_t=None,
                        v0bar_t=None, theta_bar_t=None):
    _check(lib().mdpd_window_vjp_dev(h, _tptr(xbar_t), _tptr(vbar_t), _tptr(cvir_t),
                                     _tptr(rhobar_t), _tptr(x0bar_t), _tptr(v0bar_t),
                                     _tptr(theta_bar_t)), h)


class Tuned(tuple):
    """Result of mdpd_autotune: unpacks as (density variant, [ms of NLIST,
    NLIST_THREAD]);
    .lanes is the force pass's lanes per particle, .force_ms its times at 1, 2,
    4 lanes (-1: not tried), .shape the thread-per-particle density kernel's
    code shape (MDPD_OPT_DENSITY_SHAPE) kept by the tuner."""

    def __new__(cls, chosen, ms):
        t = super().__new__(cls, (int(chosen[0]), [float(x) for x in ms[:2]]))
        t.lanes = int(chosen[1])
        t.shape = int(chosen[2])
        t.force_ms = [float(x) for x in ms[2:]]
        return t


def mdpd_autotune(h, reps: int = 5) -> Tuned:
    """Pick the faster density-pass variant, then the fastest lanes per
    particle of the force pass, on the current state."""
    chosen = np.zeros(3, np.int32)
    ms = np.zeros(5)
    _check(lib().mdpd_autotune(h, int(reps), _p(chosen), _p(ms)), h)
    return Tuned(chosen, ms)


def mdpd_density_noalloc(params, pos_t, rho_t, stream=None):
    """Densities of the particles at device positions pos_t ((n, 3) float64) into
    rho_t ((n,) float64) without any device allocation by the library (fixed
    internal scratch; n <= 65536, <= 32768 cells).  Asynchronous on `stream`."""
    cp = to_c_params(params)
    n = int(pos_t.shape[0])
    _check(lib().mdpd_density_noalloc(C.byref(cp), n, _tptr(pos_t), _tptr(rho_t),
                                      _stream_ptr(stream)))


def mdpd_measure_fma_peak():
    """(FMA lane-operations per second, best launch ms) of the current device."""
    rate, ms = C.c_double(), C.c_double()
    _check(lib().mdpd_measure_fma_peak(C.byref(rate), C.byref(ms)))
    return rate.value, ms.value


def mdpd_destroy(h):
    if h:
        lib().mdpd_destroy(h)


def mdpd_last_error(h=None) -> str:
    msg = lib().mdpd_last_error(h)
    return msg.decode() if msg else ""


class Batch:
    """Owning wrapper of a batch handle: nrep independent systems advanced by
    one launch per kernel (see ``mdpd_create_batch``)."""

    def __init__(self, params_list, n_list, pos, vel, type, seeds, stream=None):
        self.h = mdpd_create_batch(params_list, n_list, pos, vel, type, seeds, stream)
        self.n_list = [int(v) for v in n_list]
        self.offsets = np.concatenate([[0], np.cumsum(self.n_list)]).astype(int)

    @classmethod
    def from_workloads(cls, ws, stream=None, precision=None):
        ps = [w.params if precision is None else w.params.copy(precision=precision) for w in ws]
        return cls(ps, [w.n for w in ws], np.concatenate([w.pos for w in ws]),
                   np.concatenate([w.vel for w in ws]), np.concatenate([w.type for w in ws]),
                   [w.seed for w in ws], stream)

    @property
    def nrep(self) -> int:
        return len(self.n_list)

    @property
    def n(self) -> int:
        return int(self.offsets[-1])

    def step(self, nsteps: int):
        mdpd_step(self.h, nsteps)

    def sync(self):
        mdpd_sync(self.h)

    def state(self):
        return mdpd_get_state(self.h)

    def replica_state(self, r: int):
        x, v, t, rho = self.state()
        a, b = self.offsets[r], self.offsets[r + 1]
        return x[a:b], v[a:b], t[a:b], rho[a:b]

    def set_state(self, pos, vel):
        mdpd_set_state(self.h, pos, vel)

    def forces(self):
        return mdpd_forces(self.h)

    def observables(self, mean: bool = False, reset: bool = False):
        return mdpd_batch_observables(self.h, mean, reset)

    def set_params(self, params_list):
        mdpd_batch_set_params(self.h, params_list)

    def pair_count(self):
        return mdpd_pair_count(self.h)

    def set_option(self, option, value):
        mdpd_set_option(self.h, option, value)

    def profile(self):
        return mdpd_profile(self.h)

    def autotune(self, reps: int = 5):
        return mdpd_autotune(self.h, reps)

    def close(self):
        if getattr(self, "h", None):
            mdpd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class System:
    """Owning wrapper of one handle (destroyed with the object)."""

    def __init__(self, params, pos, vel, type, seed: int, stream=None):
        self.h = mdpd_create(params, pos, vel, type, seed, stream)

    @classmethod
    def from_workload(cls, w, stream=None, precision=None):
        p = w.params if precision is None else w.params.copy(precision=precision)
        s = cls(p, w.pos, w.vel, w.type, w.seed, stream)
        if w.mask is not None:
            s.set_walls(w.mask, w.voxel, w.origin, w.wall_density, w.shell, w.wall_type,
                        w.wall_seed)
        return s

    def set_walls(self, *a, **k):
        mdpd_set_walls(self.h, *a, **k)
        self.has_walls = True

    def step(self, nsteps: int):
        mdpd_step(self.h, nsteps)

    def sync(self):
        mdpd_sync(self.h)

    @property
    def n(self) -> int:
        return mdpd_num_particles(self.h)

    def state(self):
        return mdpd_get_state(self.h)

    def set_state(self, pos, vel):
        mdpd_set_state(self.h, pos, vel)

    def forces(self):
        return mdpd_forces(self.h)

    def observables(self):
        return mdpd_observables(self.h)

    def observables_mean(self, reset=True):
        return mdpd_observables_mean(self.h, reset)

    def pair_count(self):
        return mdpd_pair_count(self.h)

    def set_option(self, option, value):
        mdpd_set_option(self.h, option, value)

    def profile(self):
        return mdpd_profile(self.h)

    def wall_density(self):
        return mdpd_get_wall_density(self.h)

    def autotune(self, reps: int = 5):
        return mdpd_autotune(self.h, reps)

    def describe(self):
        return mdpd_describe(self.h)

    def close(self):
        if self.h:
            mdpd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
