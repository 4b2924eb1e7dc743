"""The allocation-free density entry point, mdpd_density_noalloc.

It serves callers that may not let the library allocate device memory (a
plugin given only its buffers by a host application that owns the device
memory, or a latency-critical path where cudaMalloc/cudaFree are not
allowed).  It keeps its temporaries in one fixed device array of the library,
so this file checks that two calls in a row -- the second one seeing the first
one's leftovers in that array -- both give the densities of Sec. 2.1 as the
FP64 oracle computes them, and the same as the allocating path
(mdpd_create + mdpd_forces); that the limits (65,536 particles, 32,768 cells)
are reached exactly and refused one step beyond; and that a particle outside
a non-periodic box is flagged with NaN.  The file is named to be collected
last.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_10134_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RHO_TOL = {0: 1e-13, 1: 2e-6}


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10134_gb300 import mdpd
    mdpd.lib()
    return torch, mdpd


def _noalloc_twice(torch, M, p, pos, stream):
    """Two calls in a row on `stream`; the inputs and outputs are made on that
    stream, so nothing else orders them."""
    out = []
    with torch.cuda.stream(stream):
        pos_t = torch.from_numpy(np.ascontiguousarray(pos)).to("cuda")
        for _ in range(2):
            rho_t = torch.full((pos.shape[0],), -1.0, dtype=torch.float64, device="cuda")
            M.mdpd_density_noalloc(p, pos_t, rho_t, stream)
            out.append(rho_t)
    stream.synchronize()
    return [r.cpu().numpy() for r in out]


def _upper_face_case():
    """A box reflecting along y with particles exactly on both y faces (the
    upper face is the edge case the binning must not lose)."""
    w = I.tiny(1800, (6.5, 5.0, 9.0), 22, periodic=(1, 0, 1))
    pos = w.pos.copy()
    pos[:40, 1] = 5.0            # on the upper face y = lo + L
    pos[40:60, 1] = 0.0          # on the lower face
    pos[60:70, 1] = np.nextafter(5.0, 0.0)
    return w.params, pos


def _limit_case():
    """Exactly the limits: 65,536 particles in a 32^3 box of 32,768 cells of
    edge r_c, non-periodic along z with particles on both z faces."""
    rng = np.random.default_rng(23)
    p = I.MDPDParams(box=(32.0, 32.0, 32.0), periodic=(1, 1, 0))
    pos = I.uniform_positions(65536, (0.0, 0.0, 0.0), (32.0, 32.0, 32.0), rng)
    pos[:64, 2] = 32.0
    pos[64:128, 2] = 0.0
    return p, pos


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_density_matches_oracle(env, precision):
    torch, M = env
    stream = torch.cuda.Stream()
    w = I.tiny(3001, (8.0, 8.0, 8.0), 21)
    cases = [("periodic", w.params, w.pos), ("upper face", *_upper_face_case()),
             ("limits", *_limit_case())]
    for name, p0, pos in cases:
        p = p0.copy(precision=precision)
        n = pos.shape[0]
        vel = np.zeros_like(pos)
        typ = np.zeros(n, np.int32)
        ref = O.Oracle(p, pos, vel, typ, 1, use_cells=n > 4000).density()
        for call, rho in enumerate(_noalloc_twice(torch, M, p, pos, stream)):
            err = np.abs(rho - ref).max()
            assert err <= RHO_TOL[precision] * ref.max(), (name, call, err)


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_density_matches_allocating_path(env, precision):
    """The same densities as the library's allocating path on inputs that
    path accepts (it refuses particles on an upper face)."""
    torch, M = env
    stream = torch.cuda.Stream()
    w1 = I.tiny(3001, (8.0, 8.0, 8.0), 21)
    w2 = I.tiny(1800, (6.5, 5.0, 9.0), 22, periodic=(1, 0, 1))
    lp, lpos = _limit_case()
    lpos = lpos.copy()
    lpos[:64, 2] = np.nextafter(32.0, 0.0)
    cases = [(w1.params, w1.pos), (w2.params, w2.pos), (lp, lpos)]
    for p0, pos in cases:
        p = p0.copy(precision=precision)
        n = pos.shape[0]
        with M.System(p, pos, np.zeros_like(pos), np.zeros(n, np.int32), 1) as s:
            _, ref = s.forces()
        for call, rho in enumerate(_noalloc_twice(torch, M, p, pos, stream)):
            assert np.abs(rho - ref).max() <= RHO_TOL[precision] * ref.max(), call


def test_noalloc_flags_particles_outside_the_box(env):
    torch, M = env
    stream = torch.cuda.Stream()
    p, pos = _upper_face_case()
    pos = pos.copy()
    pos[100, 1] = 5.25           # beyond the upper face of the reflecting axis
    pos[101, 1] = -0.5           # below the lower face
    rho = _noalloc_twice(torch, M, p.copy(precision=1), pos, stream)[1]
    assert np.isnan(rho[100]) and np.isnan(rho[101])
    assert np.all(np.isfinite(np.delete(rho, [100, 101])))


def test_noalloc_rejects_oversized_inputs(env):
    torch, M = env
    p = I.MDPDParams(box=(40.0, 40.0, 40.0))          # 64000 cells of edge rc
    pos_t = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    rho_t = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MDPDError) as e:
        M.mdpd_density_noalloc(p, pos_t, rho_t)
    assert e.value.name == "INVALID_ARG" and "cells" in str(e.value)
    p = I.MDPDParams(box=(32.0, 32.0, 33.0))          # 32 x 32 x 33 cells: one row too many
    with pytest.raises(M.MDPDError) as e:
        M.mdpd_density_noalloc(p, pos_t, rho_t)
    assert e.value.name == "INVALID_ARG"
    p = I.MDPDParams(box=(30.0, 30.0, 30.0))
    big = torch.zeros((65537, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros(65537, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MDPDError) as e:
        M.mdpd_density_noalloc(p, big, out)
    assert e.value.name == "INVALID_ARG"
