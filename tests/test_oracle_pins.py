"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, hand-worked closed forms, an independent library
routine, brute force, or a conservation law.  None needs a GPU.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_10134_gb300 import inputs as I


def _read_table(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --- Philox-4x32-10 -----------------------------------------------------------

def test_philox_known_answers(golden_dir):
    """Published known-answer vectors of Philox-4x32-10 (SC'11 / Random123)."""
    rows = _read_table(os.path.join(golden_dir, "philox4x32_10_kat.txt"))
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_xi_symmetric_and_unit_variance():
    """xi_ij = xi_ji (Sec. 2.1 needs it for momentum conservation); the uniform
    variable has mean 0, variance 1 and lies in (-sqrt3, sqrt3)."""
    rng = np.random.default_rng(5)
    vals = []
    for _ in range(4000):
        i, j = (int(x) for x in rng.integers(0, 2**32, size=2, dtype=np.uint64))
        step = int(rng.integers(0, 2**40))
        a = O.xi(7, step, i, j, 0)
        assert a == O.xi(7, step, j, i, 0)
        assert -math.sqrt(3) < a < math.sqrt(3)
        vals.append(a)
    vals = np.array(vals)
    assert abs(vals.mean()) < 4 / math.sqrt(len(vals))
    assert abs(vals.var() - 1.0) < 0.08
    # different steps and seeds give different draws
    assert O.xi(7, 1, 3, 4, 0) != O.xi(7, 2, 3, 4, 0)
    assert O.xi(7, 1, 3, 4, 0) != O.xi(8, 1, 3, 4, 0)


def test_xi_gaussian_moments():
    g = np.array([O.xi(3, s, 1, 2, 1) for s in range(20000)])
    assert abs(g.mean()) < 0.04
    assert abs(g.var() - 1.0) < 0.05
    assert abs(np.mean(g ** 4) - 3.0) < 0.25      # Gaussian kurtosis


# --- weights -----------------------------------------------------------------

@pytest.mark.parametrize("rd", [0.75, 0.5, 1.0])
def test_w_rho_normalised(rd):
    """int_0^inf 4 pi r^2 w_rho(r) dr = 1 (Sec. 2.1), by adaptive quadrature."""
    from scipy.integrate import quad
    val, err = quad(lambda r: 4 * math.pi * r * r * O.w_rho(r, rd), 0.0, rd, epsabs=1e-13)
    assert abs(val - 1.0) < 1e-10
    assert O.w_rho(rd, rd) == 0.0 and O.w_rho(1.3 * rd, rd) == 0.0


# --- single pair, worked by hand ------------------------------------------------

def test_pair_force_hand_cases(golden_dir):
    rows = _read_table(os.path.join(golden_dir, "pair_force_hand.txt"))
    for r in rows:
        name, vals = r[0], [float(x) for x in r[1:]]
        d, v = vals[0:3], vals[3:6]
        A, B, gam, ri, rj, xi = vals[6:12]
        p = I.MDPDParams()
        p.A[0, 0], p.B[0, 0], p.gamma[0, 0] = A, B, gam
        f, w = O.pair_force(p, d, v, 0, 0, ri, rj, xi)
        if math.isnan(vals[12]):
            assert f is None, name
            continue
        np.testing.assert_allclose(f, vals[12:15], rtol=1e-13, atol=1e-12, err_msg=name)
        np.testing.assert_allclose(w, vals[15:21], rtol=1e-13, atol=1e-12, err_msg=name)


def test_pair_force_antisymmetric():
    """Swapping i and j (d -> -d, v_ij -> -v_ij, same xi) flips the force:
    pairwise central forces conserve momentum."""
    rng = np.random.default_rng(2)
    p = I.MDPDParams(ntypes=3)
    for ti in range(3):
        for tj in range(ti, 3):
            p.set_pair(ti, tj, A=-50 + 20 * rng.random(), B=15 + 20 * rng.random(),
                       gamma=3 + 3 * rng.random())
    for _ in range(200):
        d = rng.uniform(-0.6, 0.6, 3)
        v = rng.normal(size=3)
        ti, tj = (int(x) for x in rng.integers(0, 3, 2))
        ri, rj, xi = 6 * rng.random(), 6 * rng.random(), rng.uniform(-1.7, 1.7)
        f1, _ = O.pair_force(p, d, v, ti, tj, ri, rj, xi)
        f2, _ = O.pair_force(p, -d, -v, tj, ti, rj, ri, xi)
        if f1 is None:
            assert f2 is None
            continue
        np.testing.assert_allclose(f1, -f2, rtol=1e-14, atol=1e-12)
        # central: parallel to d
        assert np.linalg.norm(np.cross(f1, d)) <= 1e-12 * (1 + np.linalg.norm(f1))


# --- neighbour search: cell list against brute force --------------------------------

@pytest.mark.parametrize("L,periodic,n,seed", [
    ((3.0, 3.0, 3.0), (1, 1, 1), 160, 1),      # three cells per axis: images matter
    ((3.4, 4.1, 5.3), (1, 1, 1), 300, 2),
    ((4.0, 3.0, 5.0), (1, 0, 1), 250, 3),      # a reflecting axis
    ((2.5, 3.5, 4.5), (0, 0, 0), 200, 4),      # no periodic axis, fewer than 3 cells
])
def test_cells_match_brute_force_bitwise(L, periodic, n, seed):
    w = I.tiny(n, L, seed, periodic=periodic, ntypes=2)
    a = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed, use_cells=False)
    b = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed, use_cells=True)
    assert np.array_equal(a.rho, b.rho)
    assert np.array_equal(a.a, b.a)
    assert np.array_equal(a.virial, b.virial)


def test_density_brute_force_python():
    """Density of a 40-particle box by explicit enumeration of all periodic images
    (no minimum-image shortcut), against the oracle."""
    w = I.tiny(40, (3.2, 3.0, 3.5), 9)
    o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed)
    L = np.array(w.params.box)
    rd = w.params.rd
    c = 15.0 / (2 * math.pi * rd ** 3)
    for i in range(w.n):
        acc = 0.0
        for j in range(w.n):
            if j == i:
                continue
            for sx in (-1, 0, 1):
                for sy in (-1, 0, 1):
                    for sz in (-1, 0, 1):
                        r = np.linalg.norm(w.pos[i] - w.pos[j] + L * np.array([sx, sy, sz]))
                        if r < rd:
                            acc += c * (1 - r / rd) ** 2
        assert abs(acc - o.rho[i]) <= 1e-12 * max(1.0, acc)


def test_ideal_gas_mean_density():
    """For uniformly random positions E[rho_i] = (N - 1)/V exactly (w_rho is
    normalised and j != i): an average over many boxes."""
    n, L = 200, (4.0, 4.0, 4.0)
    means = []
    for seed in range(40):
        w = I.tiny(n, L, 100 + seed)
        means.append(O.Oracle(w.params, w.pos, w.vel, w.type, w.seed).rho.mean())
    expect = (n - 1) / 64.0
    m = np.mean(means)
    sem = np.std(means) / math.sqrt(len(means))
    assert abs(m - expect) < 4 * sem + 1e-3


def test_total_force_zero():
    """With no body force and no frozen particles, sum_i F_i = 0 to round-off."""
    w = I.tiny(500, (5.0, 5.0, 5.0), 11, ntypes=3)
    o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed)
    scale = np.sqrt((o.a ** 2).sum(axis=1).mean()) * math.sqrt(w.n)
    assert np.abs(o.a.sum(axis=0)).max() < 1e-13 * scale


def test_frozen_and_body_force():
    w = I.tiny(300, (5.0, 5.0, 5.0), 12, ntypes=2)
    p = w.params.copy(frozen_types=(1,), g=(0.02, -0.01, 0.0))
    o = O.Oracle(p, w.pos, w.vel, w.type, w.seed)
    q = w.params.copy(frozen_types=(), g=(0.0, 0.0, 0.0))
    o0 = O.Oracle(q, w.pos, w.vel, w.type, w.seed)
    frozen = w.type == 1
    assert np.all(o.a[frozen] == 0.0)
    np.testing.assert_allclose(o.a[~frozen], o0.a[~frozen] + np.array([0.02, -0.01, 0.0]),
                               rtol=0, atol=1e-12)


# --- integration ---------------------------------------------------------------

def test_momentum_conserved_over_steps():
    w = I.tiny(400, (5.0, 5.0, 5.0), 13)
    o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed)
    p0 = o.v.sum(axis=0)
    o.run(50)
    assert np.abs(o.v.sum(axis=0) - p0).max() < 1e-10 * w.n


def test_zero_force_free_flight():
    """With A = B = gamma = 0 the particles fly freely: x(t) = x0 + t v0 (wrapped)."""
    w = I.tiny(100, (4.0, 4.0, 4.0), 14)
    p = w.params.copy()
    p.A[:] = 0.0
    p.B[:] = 0.0
    p.gamma[:] = 0.0
    o = O.Oracle(p, w.pos, w.vel, w.type, w.seed)
    o.run(30)
    L = np.array(p.box)
    expect = np.mod(w.pos + 30 * p.dt * w.vel, L)
    diff = (o.x - expect + L / 2) % L - L / 2
    assert np.abs(diff).max() < 1e-12
    np.testing.assert_allclose(o.v, w.vel, rtol=0, atol=1e-15)


def test_reflection_rule():
    """A drift into a solid voxel or through a reflecting face is undone and the
    half-step velocity is negated; a free drift is kept."""
    p = I.MDPDParams(box=(4.0, 4.0, 4.0), periodic=(1, 1, 0))
    p.A[:] = 0.0
    p.B[:] = 0.0
    p.gamma[:] = 0.0
    mask = np.zeros((8, 8, 8), np.uint8)
    mask[:, :, 5] = 1                                  # solid plane 2.5 <= x < 3.0
    pos = np.array([[2.49, 1.0, 1.0], [1.0, 1.0, 3.995], [1.0, 1.0, 2.0]])
    vel = np.array([[2.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.5, 0.0, 0.0]])
    o = O.Oracle(p, pos, vel, np.zeros(3, np.int32), 1, mask=mask, voxel=0.5)
    o.run(1)
    np.testing.assert_array_equal(o.x[0], pos[0])
    np.testing.assert_array_equal(o.v[0], -vel[0])
    np.testing.assert_array_equal(o.x[1], pos[1])
    np.testing.assert_array_equal(o.v[1], -vel[1])
    np.testing.assert_allclose(o.x[2], pos[2] + p.dt * vel[2], atol=1e-15)


# --- wall packing ----------------------------------------------------------------

def _shell_by_edt(mask, R, periodic):
    """Solid voxels whose Euclidean distance (voxel units) to the nearest pore
    voxel is <= R, from scipy's exact distance transform (periodic axes by
    tiling the image three times)."""
    from scipy.ndimage import distance_transform_edt
    reps = [3 if periodic[2 - k] else 1 for k in range(3)]   # mask is [z, y, x]
    tiled = np.tile(mask, reps)
    dist = distance_transform_edt(tiled != 0)
    sl = tuple(slice(mask.shape[k], 2 * mask.shape[k]) if reps[k] == 3 else slice(None)
               for k in range(3))
    return ((mask != 0) & (dist[sl] <= R + 1e-9)).astype(np.uint8)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (1, 0, 1)])
def test_wall_shell_matches_distance_transform(periodic):
    rng = np.random.default_rng(4)
    f = I.gaussian_random_field((12, 14, 16), 2.0, rng)
    mask = (f > np.quantile(f, 0.3)).astype(np.uint8)
    for shell, voxel in ((1.0, 0.5), (0.75, 0.5), (1.0, 0.25)):
        pos, sh = O.place_walls(mask, periodic, voxel, (0, 0, 0), 6.0, shell, 5)
        assert np.array_equal(sh, _shell_by_edt(mask, shell / voxel, periodic))


def test_wall_particles_inside_shell_and_density():
    rng = np.random.default_rng(6)
    f = I.gaussian_random_field((20, 20, 20), 3.0, rng)
    mask = (f > np.quantile(f, 0.4)).astype(np.uint8)
    voxel, rho_w = 0.5, 6.0
    pos, sh = O.place_walls(mask, (1, 1, 1), voxel, (0.0, 0.0, 0.0), rho_w, 1.0, 77)
    idx = np.floor(pos / voxel).astype(int)
    assert np.all(sh[idx[:, 2], idx[:, 1], idx[:, 0]] == 1)
    expect = rho_w * sh.sum() * voxel ** 3
    # per voxel the count is floor(lam + u): mean lam, variance <= 1/4
    assert abs(len(pos) - expect) < 4 * math.sqrt(0.25 * sh.sum()) + 1
    pos2, _ = O.place_walls(mask, (1, 1, 1), voxel, (0.0, 0.0, 0.0), rho_w, 1.0, 77)
    assert np.array_equal(pos, pos2)


def test_oracle_results_do_not_depend_on_thread_count():
    """Gather-only sums: densities, forces and a few steps are bit-identical
    with one thread and with all threads."""
    w = I.tiny(800, (5.0, 5.0, 5.0), 13, ntypes=2)
    n0 = O.num_threads()
    out = []
    for t in (1, n0):
        O.set_num_threads(t)
        o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed, use_cells=True)
        a, _ = o.forces()
        o.run(3)
        out.append((o.density(), a, o.x.copy()))
    O.set_num_threads(n0)
    for u, v in zip(*out):
        assert np.array_equal(u, v)
# --- the subset force routine that gives the full-size expected values -------------

# --- the subset force routine used as the checker at full size ----------------------

def _walled_rock_standin(seed):
    """A small walled porous system shaped like the rock workload: a Gaussian
    random field thresholded to pores, fluid at density 6 in the pores and
    frozen wall particles (type 1) in a 1 r_c shell, body force along x."""
    rng = np.random.default_rng(seed)
    nvox, voxel = 16, 0.5
    f = I.gaussian_random_field(nvox, 2.0, rng)
    mask = (f >= np.quantile(f, 0.35)).astype(np.uint8)
    L = nvox * voxel
    p = I.MDPDParams(box=(L, L, L), ntypes=2, g=(0.05, 0.0, 0.0), frozen_types=(1,))
    p.set_pair(0, 1, A=-30.0)
    pore = np.argwhere(mask == 0)                       # [z, y, x]
    pick = pore[rng.integers(0, len(pore), size=int(6.0 * len(pore) * voxel ** 3))]
    fluid = (pick[:, ::-1] + rng.random(pick.shape)) * voxel
    walls, _ = O.place_walls(mask, (1, 1, 1), voxel, (0.0, 0.0, 0.0), 6.0, 1.0, seed + 7)
    pos = np.concatenate([fluid, walls])
    vel = np.concatenate([I.maxwell_velocities(len(fluid), 1.0, rng), np.zeros_like(walls)])
    typ = np.concatenate([np.zeros(len(fluid), np.int32), np.ones(len(walls), np.int32)])
    return p, pos, vel, typ, mask, voxel


def _subset_cases():
    w = I.tiny(600, (5.0, 5.0, 5.0), 31, ntypes=3)
    yield "multi-type, frozen, body force", w.params.copy(
        frozen_types=(2,), g=(0.02, -0.01, 0.005)), w.pos, w.vel, w.type, {}
    w = I.tiny(500, (4.0, 3.0, 5.0), 32, periodic=(1, 0, 1), ntypes=2)
    yield "reflecting axis, Gaussian xi", w.params.copy(xi_dist=1, g=(0.0, 0.0, 0.03)), \
        w.pos, w.vel, w.type, {}
    p, pos, vel, typ, mask, voxel = _walled_rock_standin(33)
    yield "walled rock stand-in", p, pos, vel, typ, {"mask": mask, "voxel": voxel}


@pytest.mark.parametrize("use_cells", [False, True])
def test_forces_subset_equals_full_forces_bitwise(use_cells):
    """orc_forces_subset, which gives the expected values of every full-size sampled parity test,
    is a second loop over the same candidates; on every sampled particle it
    must give exactly the accelerations of orc_forces (Sec. 2.1, Eq. 1), with
    the same summation order, so the two may not differ in a single bit."""
    rng = np.random.default_rng(34)
    for name, p, pos, vel, typ, walls in _subset_cases():
        o = O.Oracle(p, pos, vel, typ, 5, use_cells=use_cells, **walls)
        o.step = 17
        rho = o.density()
        a, _ = o.forces(rho=rho, step=17)
        idx = np.concatenate([rng.choice(o.n, size=min(150, o.n), replace=False),
                              [0, o.n - 1]])
        sub = o.forces_subset(idx, rho=rho, step=17)
        assert np.array_equal(sub, a[idx]), name
        # frozen rows are zero, mobile rows carry the body force
        frozen = np.isin(typ[idx], np.array(p.frozen_types, dtype=np.int32))
        assert np.all(sub[frozen] == 0.0), name
        assert np.any(sub[~frozen] != 0.0), name
