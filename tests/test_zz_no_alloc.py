"""The allocation-free density entry point, mdpd_density_noalloc.

It serves callers that may not let the library allocate device memory (a
plugin given only its buffers by a host application that owns the device
memory, or a latency-critical path where cudaMalloc/cudaFree are not
allowed).  It keeps its temporaries in one fixed device array of the
library, so this file checks that two calls in a row -- the second one
seeing the first one's leftovers in that array -- both give the same
densities as the allocating path (mdpd_create + mdpd_forces), and that
oversized inputs are refused.  The file is named to be collected last.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_density_matches_allocating_path(env, precision):
    torch, M = env
    stream = torch.cuda.Stream()
    cases = [I.tiny(3001, (8.0, 8.0, 8.0), 21),
             I.tiny(1800, (6.5, 5.0, 9.0), 22, periodic=(1, 0, 1))]
    for w in cases:
        p = w.params.copy(precision=precision)
        with M.System(p, w.pos, w.vel, w.type, w.seed) as s:
            _, ref = s.forces()
        pos_t = torch.from_numpy(w.pos).to("cuda")
        for call in range(2):
            rho_t = torch.full((w.n,), -1.0, dtype=torch.float64, device="cuda")
            M.mdpd_density_noalloc(p, pos_t, rho_t, stream)
            stream.synchronize()
            rho = rho_t.cpu().numpy()
            assert np.abs(rho - ref).max() <= RHO_TOL[precision] * ref.max(), call


def test_noalloc_rejects_oversized_inputs(env):
    torch, M = env
    p = I.MDPDParams(box=(40.0, 40.0, 40.0))          # 64000 cells of edge rc
    pos_t = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    rho_t = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MDPDError) as e:
        M.mdpd_density_noalloc(p, pos_t, rho_t)
    assert e.value.name == "INVALID_ARG" and "cells" in str(e.value)
    p = I.MDPDParams(box=(30.0, 30.0, 30.0))
    big = torch.zeros((65537, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros(65537, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MDPDError) as e:
        M.mdpd_density_noalloc(p, big, out)
    assert e.value.name == "INVALID_ARG"
