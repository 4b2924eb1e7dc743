"""Batched replicas: many independent systems of uneven size and parameters
advanced by one launch per kernel.

The batch's contract is exact: replica r of a batch evolves bit-identically to
the same system created alone (same parameters, particles, seed and kernel
variant), because its particles keep their own slot range, its cells keep
their own order and the random stream is keyed on the index inside the
replica.  The single-system path is itself pinned to the FP64 oracle
(tests/test_gpu_parity.py); the batch's forces are also compared with the
oracle directly here.
"""
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


def replicas(precision, seed=11):
    """Five uneven replicas: different boxes, sizes, A and B, a two-type
    system, a non-periodic axis, one tiny replica (a ragged single chunk)."""
    ws = I.batch_slabs(nrep=3, n_range=(700, 2600), seed=seed, precision=precision)
    t = I.tiny(900, (4.0, 5.0, 6.5), seed + 7, periodic=(1, 0, 1), ntypes=2)
    t.params = t.params.copy(precision=precision)
    small = I.tiny(37, (3.0, 3.3, 3.1), seed + 9)
    small.params = small.params.copy(precision=precision)
    return ws[:2] + [t] + ws[2:] + [small]


def run_alone(M, w, nsteps, kernels):
    s = M.System(w.params, w.pos, w.vel, w.type, w.seed)
    s.set_option(M.OPT_KERNELS, kernels)
    s.step(nsteps)
    x, v, _, rho = s.state()
    obs = s.observables()
    s.close()
    return x, v, rho, obs


@pytest.mark.parametrize("kernels", [0, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_members_match_standalone_bitwise(M, precision, kernels):
    ws = replicas(precision)
    b = M.Batch.from_workloads(ws)
    assert b.nrep == len(ws) and M.mdpd_num_replicas(b.h) == len(ws)
    b.set_option(M.OPT_KERNELS, kernels)
    K = 25
    b.step(K)
    obs = b.observables()
    for r, w in enumerate(ws):
        x, v, t, rho = b.replica_state(r)
        xs, vs, rhos, obs_s = run_alone(M, w, K, kernels)
        assert np.array_equal(x, xs) and np.array_equal(v, vs), r
        assert np.array_equal(rho, rhos), r
        assert np.array_equal(t, w.type)
        # the observables are reduced in another order (a single system with
        # FP32 pair arithmetic adds its FP32 warp sums in FP32): equal to rounding
        tol = 1e-12 if precision == 0 else 2e-6
        assert np.allclose(obs[r], obs_s, rtol=tol, atol=tol * np.abs(obs_s).max()), r
        assert obs[r][15] == K
    b.close()


def test_batch_forces_match_oracle(M):
    ws = replicas(0, seed=5)
    b = M.Batch.from_workloads(ws)
    f, rho = b.forces()
    for r, w in enumerate(ws):
        a0, a1 = b.offsets[r], b.offsets[r + 1]
        o = O.Oracle(w.params, w.pos, w.vel, w.type, w.seed)
        ref, _ = o.forces()
        scale = max(np.sqrt((ref ** 2).sum(1).mean()), 1e-30)
        err = np.sqrt(((f[a0:a1] - ref) ** 2).sum(1)) / np.maximum(np.sqrt((ref ** 2).sum(1)), scale)
        assert err.max() <= 1e-12, (r, err.max())
        assert np.allclose(rho[a0:a1], o.density(), rtol=1e-12, atol=1e-12)
    b.close()


def test_batch_graph_direct_autotune_and_set_state(M):
    ws = replicas(1, seed=3)
    b1 = M.Batch.from_workloads(ws)
    b2 = M.Batch.from_workloads(ws)
    b2.set_option(M.OPT_GRAPH, 0)
    b1.step(12)
    b2.step(12)
    assert np.array_equal(b1.state()[0], b2.state()[0])
    # autotune keeps the state and the trajectory stays that of the chosen variant
    x0, v0, _, _ = b1.state()
    res = b1.autotune(3)
    chosen, ms = res
    assert chosen in (M.KERNELS_NLIST, M.KERNELS_NLIST_THREAD)
    assert len(ms) == 2
    assert res.lanes == 1 and res.force_ms[1:] == [-1.0, -1.0]
    x1, v1, _, _ = b1.state()
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)
    # set_state: each replica restarts from the given state (forces re-evaluated
    # with v(t), as for a single system) exactly as the same system alone does
    b2.set_state(x0, v0)
    b2.set_option(M.OPT_KERNELS, chosen)
    b2.step(5)
    for r, w in enumerate(ws):
        a0, a1 = b2.offsets[r], b2.offsets[r + 1]
        s = M.System(w.params, w.pos, w.vel, w.type, w.seed)
        s.set_option(M.OPT_KERNELS, chosen)
        s.step(12)
        s.set_state(x0[a0:a1], v0[a0:a1])
        s.step(5)
        x, v, _, _ = b2.replica_state(r)
        xs, vs, _, _ = s.state()
        assert np.array_equal(x, xs) and np.array_equal(v, vs), r
        s.close()
    b1.close()
    b2.close()


def test_batch_set_params_changes_only_that_replica(M):
    ws = replicas(1, seed=4)
    b = M.Batch.from_workloads(ws)
    b.step(3)
    ps = [w.params.copy() for w in ws]
    ps[1].set_pair(0, 0, A=-33.0, B=21.0)
    b.set_params(ps)
    b.step(6)
    alone = M.System(ws[1].params, ws[1].pos, ws[1].vel, ws[1].type, ws[1].seed)
    alone.step(3)
    M.mdpd_set_params(alone.h, ps[1])
    alone.step(6)
    x, v, _, _ = b.replica_state(1)
    xa, va, _, _ = alone.state()
    assert np.array_equal(x, xa) and np.array_equal(v, va)
    x0, _, _, _ = b.replica_state(0)
    s0 = M.System(ws[0].params, ws[0].pos, ws[0].vel, ws[0].type, ws[0].seed)
    s0.step(9)
    assert np.array_equal(x0, s0.state()[0])
    alone.close()
    s0.close()
    b.close()


def test_batch_edge_cases(M):
    ws = replicas(1, seed=6)
    # an empty replica in the middle, and a batch of one
    empty = I.tiny(0, (3.0, 3.0, 3.0), 1)
    empty.params = empty.params.copy(precision=1)
    b = M.Batch.from_workloads(ws[:2] + [empty] + ws[2:])
    b.step(4)
    obs = b.observables()
    assert np.all(obs[2][:15] == 0)
    x, _, _, _ = b.replica_state(3)
    xs, _, _, _ = run_alone(M, ws[2], 4, M.KERNELS_NLIST)
    assert np.array_equal(x, xs)
    assert b.pair_count() > 0
    with pytest.raises(M.MDPDError):
        M.mdpd_observables(b.h)
    with pytest.raises(M.MDPDError):
        M.mdpd_set_walls(b.h, np.ones((4, 4, 4), np.uint8), 0.5, (0, 0, 0), 6.0, 1.0, 0, 1)
    with pytest.raises(M.MDPDError):
        b.set_option(M.OPT_KERNELS, M.KERNELS_SCAN)
    b.close()
    one = M.Batch.from_workloads(ws[:1])
    one.step(7)
    xs, vs, _, _ = run_alone(M, ws[0], 7, M.KERNELS_NLIST)
    assert np.array_equal(one.state()[0], xs)
    one.close()
    # invalid batches
    with pytest.raises(M.MDPDError):
        M.Batch([], [], np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.int32), [])
    mixed = [ws[0].params.copy(precision=0), ws[1].params]
    with pytest.raises(M.MDPDError):
        M.Batch(mixed, [ws[0].n, ws[1].n], np.concatenate([ws[0].pos, ws[1].pos]),
                np.concatenate([ws[0].vel, ws[1].vel]), np.zeros(ws[0].n + ws[1].n, np.int32),
                [1, 2])
    bad_type = np.zeros(ws[0].n + ws[1].n, np.int32)
    bad_type[ws[0].n + 3] = 1                         # replica 1 has one type
    with pytest.raises(M.MDPDError):
        M.Batch([ws[0].params, ws[1].params], [ws[0].n, ws[1].n],
                np.concatenate([ws[0].pos, ws[1].pos]), np.concatenate([ws[0].vel, ws[1].vel]),
                bad_type, [1, 2])


def test_uneven_batch_sampled_members(M):
    """A 64-replica batch of the slab family (N_r from 2k to 20k): three
    members, the smallest, the largest and one in between, are bit-identical
    to their standalone runs; every replica reports finite observables and
    its own step count."""
    ws = I.batch_slabs(nrep=64, seed=2, precision=1)
    b = M.Batch.from_workloads(ws)
    b.step(30)
    ns = np.array([w.n for w in ws])
    for r in (int(ns.argmin()), int(ns.argmax()), 17):
        x, v, _, _ = b.replica_state(r)
        xs, vs, _, _ = run_alone(M, ws[r], 30, M.KERNELS_NLIST)
        assert np.array_equal(x, xs) and np.array_equal(v, vs), r
    obs = b.observables()
    assert np.all(np.isfinite(obs)) and np.all(obs[:, 15] == 30)
    assert np.array_equal(obs[:, 14], ns.astype(float))      # mobile count per replica
    b.close()


def test_full_batch_sampled_parity(M):
    """The full 256-replica batch as the bench runs it (FP32, autotuned, a few
    steps): for four replicas (smallest, largest, two others) the densities
    of all their particles and the forces of a sample equal the oracle's at
    the same state and step index."""
    import math
    ws = I.batch_slabs(nrep=256, seed=1, precision=1)
    b = M.Batch.from_workloads(ws)
    b.autotune()
    b.step(5)
    f, rho = b.forces()
    x, v, t, _ = b.state()
    ns = np.array([w.n for w in ws])
    for r in (int(ns.argmin()), int(ns.argmax()), 77, 200):
        a0, a1 = b.offsets[r], b.offsets[r + 1]
        w = ws[r]
        o = O.Oracle(w.params.copy(precision=0), x[a0:a1], v[a0:a1], t[a0:a1], w.seed,
                     use_cells=True)
        assert np.abs(rho[a0:a1] - o.rho).max() <= 2e-6 * o.rho.max(), r
        idx = np.random.default_rng(r).choice(a1 - a0, min(200, a1 - a0), replace=False)
        ref = o.forces_subset(idx, rho=o.rho, step=5)
        rms = math.sqrt(np.mean(np.sum(ref ** 2, axis=1)))
        err = np.linalg.norm(f[a0:a1][idx] - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), rms)
        assert err.max() <= 1e-5, (r, err.max())
    b.close()
