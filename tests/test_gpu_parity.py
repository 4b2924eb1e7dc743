"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Tolerances (per particle, ||f_gpu - f_ora|| / max(||f_ora||, rms f)):
FP64 pair arithmetic 1e-12, FP32 pair arithmetic 1e-5.  Integer and index
results (wall placement counts, ids, types) are compared exactly.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_10134_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}
RHO_TOL = {0: 1e-13, 1: 2e-6}


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10134_gb300 import mdpd
    mdpd.lib()
    return mdpd


def rel_force_err(f, ref):
    nrm = np.linalg.norm(ref, axis=1)
    rms = math.sqrt(np.mean(nrm ** 2)) if len(nrm) else 1.0
    den = np.maximum(nrm, rms)
    return (np.linalg.norm(f - ref, axis=1) / den).max() if len(f) else 0.0


def make(M, w, precision):
    p = w.params.copy(precision=precision)
    return M.System(p, w.pos, w.vel, w.type, w.seed), p


CASES = [
    # n, box, periodic, ntypes, seed
    (3001, (8.0, 8.0, 8.0), (1, 1, 1), 1, 1),          # several blocks + ragged tail
    (1500, (3.0, 9.0, 7.3), (1, 1, 1), 3, 2),          # 3 cells on x: images
    (2200, (6.5, 5.0, 9.0), (1, 0, 1), 2, 3),          # reflecting y faces
    (700, (2.4, 4.0, 3.5), (0, 0, 0), 2, 4),           # no periodic axis, nc < 3
]


# (kernel variant, code shape of the thread-per-particle density kernel)
VARIANTS = [(0, 0), (1, 0), (2, 0), (2, 1)]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", CASES)
def test_forces_and_density_match_oracle(M, case, precision, variant):
    n, L, per, nt, seed = case
    w = I.tiny(n, L, seed, periodic=per, ntypes=nt, g=(0.01, -0.02, 0.005),
               frozen_types=(1,) if nt > 1 else ())
    s, p = make(M, w, precision)
    s.set_option(M.OPT_KERNELS, variant[0])
    s.set_option(M.OPT_DENSITY_SHAPE, variant[1])
    f, rho = s.forces()
    o = O.Oracle(p, w.pos, w.vel, w.type, w.seed)
    assert np.abs(rho - o.rho).max() <= RHO_TOL[precision] * max(1.0, o.rho.max())
    assert rel_force_err(f, o.a) <= TOL[precision]
    obs = s.observables()
    ref = o.observables()
    scale = np.abs(ref[5:8]).max()
    assert np.abs(obs[5:11] - ref[5:11]).max() <= (1e-11 if precision == 0 else 1e-5) * scale
    assert obs[14] == ref[14]
    _, _, typ, rho2 = s.state()
    assert np.array_equal(typ, w.type)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_gaussian_xi_and_rho_self(M, precision):
    w = I.tiny(1200, (6.0, 6.0, 6.0), 8, ntypes=2, xi_dist=1, rho_self=1)
    s, p = make(M, w, precision)
    f, rho = s.forces()
    o = O.Oracle(p, w.pos, w.vel, w.type, w.seed)
    assert np.abs(rho - o.rho).max() <= RHO_TOL[precision] * o.rho.max()
    # Box-Muller goes through log/cos: allow the library functions' rounding
    assert rel_force_err(f, o.a) <= (1e-11 if precision == 0 else 2e-5)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_short_trajectory_matches_oracle(M, precision):
    w = I.tiny(2500, (7.0, 7.0, 7.0), 5, ntypes=2, g=(0.05, 0.0, 0.0))
    s, p = make(M, w, precision)
    o = O.Oracle(p, w.pos, w.vel, w.type, w.seed)
    for _ in range(3):
        s.step(4)
        o.run(4)
        x, v, _, rho = s.state()
        L = np.array(p.box)
        dx = (x - o.x + L / 2) % L - L / 2
        # FP32 forces agree to ~1e-5 of rms f; over a few steps that moves v by
        # ~dt * 1e-5 * |f| per half-kick and x by dt times that
        tol_x = 1e-12 if precision == 0 else 2e-5
        tol_v = 1e-10 if precision == 0 else 5e-4
        assert np.abs(dx).max() < tol_x
        assert np.abs(v - o.v).max() < tol_v * max(1.0, np.abs(o.v).max())
    obs = s.observables()
    ref = o.observables()
    np.testing.assert_allclose(obs[:3], ref[:3], atol=1e-9 if precision == 0 else 2e-2)
    np.testing.assert_allclose(obs[3:5], ref[3:5], rtol=1e-10 if precision == 0 else 1e-4)
    np.testing.assert_allclose(obs[5:11], ref[5:11], rtol=1e-9 if precision == 0 else 1e-4,
                               atol=1e-6 if precision == 0 else 1e-2)
    assert obs[14] == ref[14] and obs[15] == ref[15] == 12
    s.close()


def test_walls_placement_and_reflection_match_oracle(M):
    rng = np.random.default_rng(3)
    nvox = (20, 16, 24)              # [z, y, x]
    voxel = 0.5
    f = I.gaussian_random_field(nvox, 2.5, rng)
    mask = (f > np.quantile(f, 0.45)).astype(np.uint8)
    L = (nvox[2] * voxel, nvox[1] * voxel, nvox[0] * voxel)
    p = I.MDPDParams(box=L, periodic=(1, 1, 1), ntypes=2, frozen_types=(1,), g=(0.1, 0, 0),
                     precision=0)
    p.set_pair(0, 1, A=-30.0)
    pore = np.flatnonzero(mask.reshape(-1) == 0)
    npart = 800
    pick = pore[rng.integers(0, pore.size, npart)]
    idx = np.stack([pick % nvox[2], (pick // nvox[2]) % nvox[1], pick // (nvox[2] * nvox[1])], 1)
    pos = (idx + rng.random((npart, 3))) * voxel
    vel = I.maxwell_velocities(npart, 1.0, rng)
    typ = np.zeros(npart, np.int32)
    s = M.System(p, pos, vel, typ, 9)
    s.set_walls(mask, voxel, (0.0, 0.0, 0.0), 6.0, 1.0, 1, 77)
    wpos, _ = O.place_walls(mask, (1, 1, 1), voxel, (0.0, 0.0, 0.0), 6.0, 1.0, 77)
    x, v, t, rho = s.state()
    assert x.shape[0] == npart + wpos.shape[0]
    assert np.array_equal(x[npart:], wpos)            # same FP64 operations: bit-exact
    assert np.all(t[npart:] == 1) and np.all(v[npart:] == 0)
    allpos = np.concatenate([pos, wpos])
    alltyp = np.concatenate([typ, np.ones(len(wpos), np.int32)])
    allvel = np.concatenate([vel, np.zeros_like(wpos)])
    o = O.Oracle(p, allpos, allvel, alltyp, 9, mask=mask, voxel=voxel)
    f, _ = s.forces()
    assert rel_force_err(f, o.a) <= 1e-12
    s.step(10)
    o.run(10)
    x, v, _, _ = s.state()
    Lv = np.array(L)
    dx = (x - o.x + Lv / 2) % Lv - Lv / 2
    assert np.abs(dx).max() < 1e-11
    assert np.abs(v - o.v).max() < 1e-9
    # nothing entered a solid voxel
    q = np.floor(x[:npart] / voxel).astype(int)
    assert np.all(mask[q[:, 2], q[:, 1], q[:, 0]] == 0)
    s.close()


def test_graph_and_direct_launch_agree_bitwise(M):
    w = I.tiny(4000, (9.0, 9.0, 9.0), 6)
    a = M.System(w.params.copy(precision=1), w.pos, w.vel, w.type, 3)
    b = M.System(w.params.copy(precision=1), w.pos, w.vel, w.type, 3)
    b.set_option(M.OPT_GRAPH, 0)
    a.step(7)
    b.step(7)
    xa, va, _, ra = a.state()
    xb, vb, _, rb = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ra, rb)
    a.step(5)
    a2 = a.state()
    # rerun from scratch: deterministic
    c = M.System(w.params.copy(precision=1), w.pos, w.vel, w.type, 3)
    c.step(12)
    assert np.array_equal(c.state()[0], a2[0])
    for s in (a, b, c):
        s.close()


def test_set_state_roundtrip_and_resume(M):
    w = I.tiny(1800, (6.0, 6.0, 6.0), 7)
    p = w.params.copy(precision=0)
    a = M.System(p, w.pos, w.vel, w.type, 5)
    a.step(6)
    x, v, _, _ = a.state()
    b = M.System(p, w.pos, w.vel, w.type, 5)
    b.set_state(x, v)
    fa, ra = a.forces()
    fb, rb = b.forces()
    # b's step index is 0, a's is 6: densities agree, forces differ only by the draw
    assert np.abs(ra - rb).max() < 1e-13
    a.close()
    b.close()


def test_degenerate_inputs(M):
    p = I.MDPDParams(box=(4.0, 4.0, 4.0), precision=0)
    # empty system
    s = M.System(p, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.int32), 1)
    s.step(3)
    assert s.state()[0].shape == (0, 3)
    s.close()
    # one particle: no neighbours, free flight
    s = M.System(p, [[1.0, 1.0, 1.0]], [[0.5, 0.0, -0.25]], [0], 1)
    f, rho = s.forces()
    assert np.all(f == 0) and rho[0] == 0
    s.step(10)
    np.testing.assert_allclose(s.state()[0][0], [1.05, 1.0, 0.975], atol=1e-14)
    s.close()
    # coincident pair: density counts w_rho(0) each, the force skips r = 0
    pos = np.array([[2.0, 2.0, 2.0], [2.0, 2.0, 2.0], [2.6, 2.0, 2.0]])
    s = M.System(p, pos, np.zeros((3, 3)), np.zeros(3, np.int32), 1)
    f, rho = s.forces()
    o = O.Oracle(p, pos, np.zeros((3, 3)), np.zeros(3, np.int32), 1)
    np.testing.assert_allclose(rho, o.rho, rtol=1e-14)
    np.testing.assert_allclose(f, o.a, rtol=1e-12, atol=1e-12)
    s.close()
    # pair exactly at r_c: no interaction
    pos = np.array([[1.0, 1.0, 1.0], [2.0, 1.0, 1.0]])
    s = M.System(p, pos, np.zeros((2, 3)), np.zeros(2, np.int32), 1)
    f, rho = s.forces()
    assert np.all(f == 0)
    s.close()


def test_nonfinite_input_is_reported(M):
    w = I.tiny(50, (4.0, 4.0, 4.0), 1)
    pos = w.pos.copy()
    pos[7, 1] = np.nan
    with pytest.raises(M.MDPDError) as e:
        M.System(w.params, pos, w.vel, w.type, 1)
    assert e.value.name == "NONFINITE"


@pytest.mark.parametrize("name", ["bulk", "slab"])
def test_workload_sampled_parity(M, name):
    """Full-size paper-shaped workloads, FP32 as benchmarked: forces of a
    sample of particles against the oracle, densities of all particles."""
    w = I.bulk() if name == "bulk" else I.slab()
    s, p = make(M, w, 1)
    f, rho = s.forces()
    o = O.Oracle(p, w.pos, w.vel, w.type, w.seed, use_cells=True)
    assert np.abs(rho - o.rho).max() <= RHO_TOL[1] * o.rho.max()
    idx = np.random.default_rng(0).choice(w.n, 400, replace=False)
    ref = o.forces_subset(idx, rho=o.rho)
    rms = math.sqrt(np.mean(np.sum(o.a ** 2, axis=1)))
    err = np.linalg.norm(f[idx] - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), rms)
    assert err.max() <= TOL[1]
    s.close()


@pytest.mark.parametrize("variant", [(0, 0), (2, 0), (2, 1)])
@pytest.mark.parametrize("precision", [0, 1])
def test_dense_particles_overflow_the_list(M, precision, variant):
    """At density ~47 every particle has ~200 partners within r_c, more than the
    64 list slots: the force pass falls back to scanning the cells itself."""
    w = I.tiny(3000, (4.0, 4.0, 4.0), 31, ntypes=2, spread=0.5)
    s, p = make(M, w, precision)
    s.set_option(M.OPT_KERNELS, variant[0])
    s.set_option(M.OPT_DENSITY_SHAPE, variant[1])
    f, rho = s.forces()
    o = O.Oracle(p, w.pos, w.vel, w.type, w.seed)
    assert np.abs(rho - o.rho).max() <= RHO_TOL[precision] * o.rho.max()
    assert rel_force_err(f, o.a) <= TOL[precision]
    assert s.pair_count() > 64 * w.n
    s.close()


def test_list_and_scan_kernels_agree(M):
    w = I.tiny(5000, (9.5, 9.0, 10.0), 32, ntypes=2, g=(0.02, 0, 0))
    a = M.System(w.params.copy(precision=1), w.pos, w.vel, w.type, 3)
    b = M.System(w.params.copy(precision=1), w.pos, w.vel, w.type, 3)
    b.set_option(M.OPT_KERNELS, M.KERNELS_SCAN)
    b.set_state(w.pos, w.vel)
    a.step(20)
    b.step(20)
    xa, va, _, ra = a.state()
    xb, vb, _, rb = b.state()
    L = np.array(w.params.box)
    # same pairs, same per-pair arithmetic; only the order of the FP32 sums differs
    assert np.abs((xa - xb + L / 2) % L - L / 2).max() < 1e-5
    assert np.abs(ra - rb).max() < 1e-4
    assert a.pair_count() == b.pair_count()
    a.close()
    b.close()


def test_autotune_keeps_state_and_parity(M):
    w = I.tiny(4000, (9.0, 9.0, 9.0), 41, ntypes=2)
    p = w.params.copy(precision=0)
    s = M.System(p, w.pos, w.vel, w.type, w.seed)
    s.step(3)
    x0, v0, _, _ = s.state()
    res = s.autotune(reps=3)
    chosen, ms = res
    assert chosen in (M.KERNELS_NLIST, M.KERNELS_NLIST_THREAD)
    assert len(ms) == 2 and min(ms) > 0
    assert res.lanes in (1, 2, 4) and len(res.force_ms) == 3 and min(res.force_ms) > 0
    x1, v1, _, _ = s.state()
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)
    o = O.Oracle(p, w.pos, w.vel, w.type, w.seed)
    o.run(3)
    f, rho = s.forces()
    a, _ = o.forces()
    assert rel_force_err(f, a) <= TOL[0]
    s.close()


def test_sampled_profile_counts(M):
    w = I.tiny(3000, (8.0, 8.0, 8.0), 42)
    s = M.System(w.params.copy(precision=1), w.pos, w.vel, w.type, 1)
    s.set_option(M.OPT_PROFILE, 100)
    s.set_option(M.OPT_PROFILE_EVERY, 4)
    s.step(20)
    prof, steps, launches = s.profile()
    assert steps == 5
    _, lps = s.describe()
    assert launches == 20 * lps          # the first half-kick rides on the binning
    assert all(v > 0 for v in prof.values())
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["slit", "rock"])
def test_wall_density_matches_oracle(M, name, precision):
    """Wall-particle density phi (Sec. 3.2, Algorithm 1) accumulated in the
    density pass: equal to the oracle's on the same positions (FP64 1e-12,
    FP32 2e-5 (1 + phi)); the option changes nothing else (the trajectory is
    bit-identical with it on and off, on the same density variant), and reading
    phi with it off is an error."""
    if name == "slit":
        w = I.slit(Lx=6.0, Ly=6.0, H=6.0, wall=1.0, voxel=0.5, g=0.2, seed=3, precision=precision)
    else:
        w = I.rock(nvox=32, voxel=0.5, corr=4.0, porosity=0.3, g=0.5, seed=5, precision=precision)
    s_on = M.System.from_workload(w, precision=precision)
    s_off = M.System.from_workload(w, precision=precision)
    # phi rides on the thread-per-particle density pass: compare with that variant
    s_off.set_option(M.OPT_KERNELS, M.KERNELS_NLIST_THREAD)
    with pytest.raises(M.MDPDError):
        s_on.wall_density()
    s_on.set_option(M.OPT_WALL_DENSITY, 1)
    tol = 1e-12 if precision == 0 else 2e-5
    for k in range(3):
        if k == 0:
            s_on.forces()
        else:
            s_on.step(7)
            s_off.step(7)
        phi = s_on.wall_density()
        x, v, t, _ = s_on.state()
        o = O.Oracle(w.params.copy(precision=0), x, v, t, w.seed, use_cells=True)
        ref = o.wall_density()
        assert np.all(ref[t == w.wall_type] == 0) and np.all(phi[t == w.wall_type] == 0)
        assert ref[t != w.wall_type].max() > 1.0          # particles do sit near walls
        assert np.all(np.abs(phi - ref) <= tol * (1 + np.abs(ref))), np.abs(phi - ref).max()
        if k > 0:
            xo, vo, _, _ = s_off.state()
            assert np.array_equal(x, xo) and np.array_equal(v, vo)
    s_on.set_option(M.OPT_WALL_DENSITY, 0)
    s_on.step(1)
    with pytest.raises(M.MDPDError):
        s_on.wall_density()
    s_on.close()
    s_off.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_split_and_fused_steps_agree_bitwise(M, precision):
    """step(3) + step(2) + step(4) gives the same trajectory, bit for bit, as
    step(9): the last step of a call stores v(t + dt) and a(t + dt), and the
    next call's first half-kick repeats exactly the arithmetic that a fused
    step performs."""
    w = I.tiny(2200, (7.0, 6.5, 7.5), 19, ntypes=2, g=(0.03, 0.0, 0.0))
    a, _ = make(M, w, precision)
    b, _ = make(M, w, precision)
    a.step(9)
    for k in (3, 2, 4):
        b.step(k)
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    a.close()
    b.close()


def test_fma_peak_is_plausible(M):
    """The measured FP32 issue rate (the ALU roofline's denominator) lies
    between half and 1.1 times the nominal 128 lanes per SM per clock at the
    maximum SM clock of this part (2.07 GHz)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * 2.07e9
    rate, ms = M.mdpd_measure_fma_peak()
    assert ms > 0
    assert 0.5 * nominal < rate < 1.1 * nominal, (rate, nominal)


@pytest.mark.parametrize("precision", [0, 1])
def test_multi_step_graph_matches_direct_launches(M, precision):
    """step(37) replays 8-step graphs for the middle of the call; the
    trajectory equals direct launches bit for bit, and the launch count is
    unchanged."""
    w = I.tiny(2500, (7.0, 7.5, 6.5), 29, ntypes=2)
    a, _ = make(M, w, precision)
    b, _ = make(M, w, precision)
    b.set_option(M.OPT_GRAPH, 0)
    for s in (a, b):
        s.set_option(M.OPT_PROFILE, 0)
        s.step(37)
        s.step(11)
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.observables(), b.observables())
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_resume_is_bitwise(M, precision):
    """A run checkpointed after 20 steps (positions, velocities, the stored
    accelerations, the step count, the seed) and resumed in a new handle
    continues bit for bit; plain set_state (forces re-evaluated with v(t))
    does not, which is why the accelerations are part of the checkpoint."""
    w = I.tiny(2000, (7.0, 6.0, 6.5), 33, ntypes=2, g=(0.02, 0.0, 0.0))
    a, p = make(M, w, precision)
    a.step(20)
    x, v, _, _ = a.state()
    acc = M.mdpd_get_accel(a.h)
    steps = M.mdpd_step_count(a.h)
    assert steps == 20
    b = M.System(p, w.pos, w.vel, w.type, w.seed)
    M.mdpd_set_step(b.h, steps)
    M.mdpd_set_state_accel(b.h, x, v, acc)
    a.step(15)
    b.step(15)
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    c = M.System(p, w.pos, w.vel, w.type, w.seed)
    M.mdpd_set_step(c.h, steps)
    c.set_state(x, v)
    c.step(15)
    assert not np.array_equal(c.state()[1], va)
    for s in (a, b, c):
        s.close()


def _rock_thread(M, precision, seed=5):
    w = I.rock(nvox=32, voxel=0.5, corr=4.0, porosity=0.3, g=0.5, seed=seed, precision=precision)
    s = M.System.from_workload(w, precision=precision)
    s.set_option(M.OPT_KERNELS, M.KERNELS_NLIST_THREAD)
    return w, s


@pytest.mark.parametrize("precision", [0, 1])
def test_frozen_split_density_tracks_oracle(M, precision):
    """With frozen wall particles the thread-per-particle density pass scans
    only the mobile candidates of a frozen home and adds the home's
    frozen-frozen part, computed once: the densities of all particles (fluid
    and wall) stay equal to the oracle's as the fluid moves."""
    w, s = _rock_thread(M, precision)
    nwall = 0
    for k in range(3):
        s.step(6)
        x, v, t, rho = s.state()
        nwall = int(np.sum(t == w.wall_type))
        o = O.Oracle(w.params.copy(precision=0), x, v, t, w.seed, use_cells=True)
        err = np.abs(rho - o.rho)
        assert err.max() <= RHO_TOL[precision] * max(1.0, o.rho.max()), err.max()
    assert nwall > 1000                      # the split had frozen homes to work on
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_frozen_split_graph_direct_and_resume_bitwise(M, precision):
    """On a walled system with the split density pass: graph replay equals
    direct launches bit for bit, and a checkpoint resumed in a new handle
    (whose frozen-frozen densities are recomputed there) continues bit for
    bit."""
    w, a = _rock_thread(M, precision)
    _, b = _rock_thread(M, precision)
    b.set_option(M.OPT_GRAPH, 0)
    for s in (a, b):
        s.step(19)
    xa, va, _, ra = a.state()
    xb, vb, _, rb = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ra, rb)
    acc = M.mdpd_get_accel(a.h)
    steps = M.mdpd_step_count(a.h)
    _, c = _rock_thread(M, precision)
    M.mdpd_set_step(c.h, steps)
    M.mdpd_set_state_accel(c.h, xa, va, acc)
    a.step(11)
    c.step(11)
    xa, va, _, ra = a.state()
    xc, vc, _, rc = c.state()
    assert np.array_equal(xa, xc) and np.array_equal(va, vc) and np.array_equal(ra, rc)
    for s in (a, b, c):
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["rock", "tiny", "dense"])
def test_density_code_shapes_agree_bitwise(M, name, precision):
    """The two code shapes of the thread-per-particle density kernel compute
    the same arithmetic: trajectories agree bit for bit, also in a dense box
    (about 200 partners per particle, beyond the list slots)."""
    if name == "rock":
        runs = [_rock_thread(M, precision)[1] for _ in range(2)]
    else:
        if name == "tiny":
            w = I.tiny(3000, (8.0, 7.0, 7.5), 41, ntypes=2, g=(0.02, 0.0, 0.0))
        else:
            w = I.tiny(3000, (4.0, 4.0, 4.0), 31, ntypes=2, spread=0.5)
        runs = [make(M, w, precision)[0] for _ in range(2)]
        for s in runs:
            s.set_option(M.OPT_KERNELS, M.KERNELS_NLIST_THREAD)
    for k, s in enumerate(runs):
        s.set_option(M.OPT_DENSITY_SHAPE, k)
    with pytest.raises(M.MDPDError):
        runs[0].set_option(M.OPT_DENSITY_SHAPE, 2)
    for s in runs:
        s.step(12)
    xa, va, _, ra = runs[0].state()
    for s in runs[1:]:
        xb, vb, _, rb = s.state()
        assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ra, rb)
    for s in runs:
        s.close()


@pytest.mark.parametrize("name", ["rock", "slit", "rock338"])
def test_full_walled_workload_sampled_parity(M, name):
    """The full-size walled workloads as the bench runs them (FP32, kernels
    picked by the autotuner, frozen split on, a few fused steps): after the
    steps, the densities of all particles (fluid and wall) and the forces of
    a sample of 400 fluid particles at the current step index equal the
    oracle's at the same state.  rock338 is the 10M-particle rock (a 38.6M
    voxel image, walls placed by the segmented scan)."""
    w = I.rock() if name == "rock" else (I.rock(nvox=338) if name == "rock338" else I.slit())
    s = M.System.from_workload(w, precision=1)
    s.autotune()
    s.step(5)
    x, v, t, rho = s.state()
    k = M.mdpd_step_count(s.h)
    assert k == 5
    f, rho_e = s.forces()                     # evaluation at the current state, step index k
    assert np.array_equal(rho, rho_e)
    p = w.params.copy(precision=0)
    o = O.Oracle(p, x, v, t, w.seed, use_cells=True)
    assert np.abs(rho - o.rho).max() <= RHO_TOL[1] * o.rho.max()
    mobile = np.flatnonzero(t != w.wall_type)
    idx = np.random.default_rng(1).choice(mobile, 400, replace=False)
    ref = o.forces_subset(idx, rho=o.rho, step=k)
    rms = math.sqrt(np.mean(np.sum(ref ** 2, axis=1)))
    err = np.linalg.norm(f[idx] - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), rms)
    assert err.max() <= TOL[1], err.max()
    assert np.all(f[t == w.wall_type] == 0)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_set_state_with_moved_walls_recomputes_frozen_part(M, precision):
    """set_state keeps the frozen-frozen density part only while every frozen
    particle is loaded at the bits it was computed from: one wall particle
    moved by a small step changes the walls' densities, which then equal the
    oracle's at the new state; loading the state unchanged keeps them."""
    w, s = _rock_thread(M, precision)
    s.step(4)
    x, v, t, _ = s.state()
    acc = M.mdpd_get_accel(s.h)
    walls = np.flatnonzero(t == w.wall_type)
    x2 = x.copy()
    x2[walls[len(walls) // 2]] += np.array([0.05, -0.03, 0.02])
    for xs in (x, x2, x2, x):
        M.mdpd_set_state_accel(s.h, xs, v, acc)
        f, rho = s.forces()
        o = O.Oracle(w.params.copy(precision=0), xs, v, t, w.seed, use_cells=True,
                     step=M.mdpd_step_count(s.h))
        assert np.abs(rho - o.rho).max() <= RHO_TOL[precision] * max(1.0, o.rho.max())
        mob = t != w.wall_type
        assert rel_force_err(f[mob], o.a[mob]) <= TOL[precision]
    s.close()


def test_loaded_positions_wrap_like_the_periodic_rule(M):
    """Positions loaded on a periodic axis are wrapped by x - L floor((x -
    lo) / L), and onto lo if the result leaves [lo, hi): in-box positions
    (also those just below hi, where x - lo can round to L) keep their bits.
    Checked against the same FP64 rule in numpy, on a box with lo != 0, for
    positions at most one box length out (there L * floor(...) is exact, so
    the rule has one rounding however the product and difference are
    contracted)."""
    lo = np.array([-3.3, 0.7, -100.1])
    L = np.array([7.3, 6.0, 9.9])
    hi = lo + L
    p = I.MDPDParams(box_lo=tuple(lo), box=tuple(L))
    rng = np.random.default_rng(8)
    x = lo + rng.random((600, 3)) * L
    k = 0
    for ax in range(3):
        for val in (lo[ax], np.nextafter(lo[ax], np.inf), np.nextafter(lo[ax], -np.inf),
                    hi[ax], np.nextafter(hi[ax], -np.inf),
                    np.nextafter(np.nextafter(hi[ax], -np.inf), -np.inf),
                    hi[ax] + 0.25 * L[ax], lo[ax] - 0.25 * L[ax], lo[ax] - 0.75 * L[ax]):
            x[k, ax] = val
            k += 1
    want = x.copy()
    for ax in range(3):
        c = want[:, ax]
        wv = np.floor((c - lo[ax]) / L[ax])
        c = np.where(wv != 0.0, c - L[ax] * wv, c)
        c = np.where((c >= hi[ax]) | (c < lo[ax]), lo[ax], c)
        want[:, ax] = c
    n = x.shape[0]
    with M.System(p, lo + 0.5 * L + np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n, np.int32), 3) as s:
        M.mdpd_set_state_accel(s.h, x, np.zeros((n, 3)), np.zeros((n, 3)))
        got = s.state()[0]
    assert np.array_equal(got.view(np.int64), want.view(np.int64))


def test_walls_from_a_mask_beyond_one_scan(M):
    """A voxel image of more voxels (264 x 264 x 256 = 17.8M) than one
    two-level scan covers (16.7M): the wall counts are scanned in segments
    joined by a running carry, and the wall particles equal the oracle's
    placement bit for bit (same ids by ascending voxel id).  The solid part
    is two slabs, one of them at the far end of the image, whose shell
    particles come after the segment boundary."""
    nvox = (256, 264, 264)           # [z, y, x]
    voxel = 0.5
    mask = np.zeros(nvox, np.uint8)
    mask[:6] = 1                     # z < 3: lower wall
    mask[250:] = 1                   # z >= 125: upper wall (voxels beyond 16.7M)
    L = (nvox[2] * voxel, nvox[1] * voxel, nvox[0] * voxel)
    p = I.MDPDParams(box=L, periodic=(1, 1, 1), ntypes=2, frozen_types=(1,), precision=1)
    rng = np.random.default_rng(12)
    npart = 2000
    pos = np.stack([rng.random(npart) * L[0], rng.random(npart) * L[1],
                    3.5 + rng.random(npart) * 120.0], 1)
    vel = I.maxwell_velocities(npart, 1.0, rng)
    with M.System(p, pos, vel, np.zeros(npart, np.int32), 4) as s:
        s.set_walls(mask, voxel, (0.0, 0.0, 0.0), 6.0, 1.0, 1, 5)
        wpos, _ = O.place_walls(mask, (1, 1, 1), voxel, (0.0, 0.0, 0.0), 6.0, 1.0, 5)
        x, _, t, _ = s.state()
    assert np.prod(nvox) > 4096 * 4096
    assert x.shape[0] == npart + wpos.shape[0] and wpos.shape[0] > 100000
    assert np.array_equal(x[npart:], wpos)
    assert np.all(t[npart:] == 1)
