"""The index-checking debug build (libmdpd_gb300_debug.so, -DMDPD_DEBUG).

Its kernels check every computed neighbour-cell range and partner index
against the arrays (a failed check sets a status bit, reported as
MDPD_ERR_BOUNDS, and skips the access).  Run in a child process with
MDPD_DEBUG=1 on a walled system (both density variants and the frozen
split), a batch of replicas and the adjoint, it must report no failed check
and give results bit-identical to the release build: the checks change no
arithmetic.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1903_10134_gb300 import inputs as I

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def run_cases(out_path):
    """The workloads of this file; results saved to out_path (npz)."""
    import torch
    from paper_1903_10134_gb300 import adjoint as AD, mdpd as M
    res = {}
    w = I.slit(Lx=8.0, Ly=8.0, H=6.0, wall=1.0, voxel=0.5, g=0.2, seed=3, precision=1)
    for k, kern in enumerate((M.KERNELS_NLIST, M.KERNELS_NLIST_THREAD, M.KERNELS_SCAN)):
        s = M.System.from_workload(w)
        s.set_option(M.OPT_KERNELS, kern)
        s.step(20)
        x, v, _, rho = s.state()
        f, r2 = s.forces()
        res[f"slit{k}_x"], res[f"slit{k}_v"], res[f"slit{k}_f"] = x, v, f
        res[f"slit{k}_rho"] = r2
        s.close()
    ws = I.batch_slabs(nrep=6, n_range=(300, 900), seed=4, precision=1)
    b = M.Batch.from_workloads(ws)
    b.step(15)
    res["batch_x"] = b.state()[0]
    res["batch_obs"] = b.observables()
    abar = torch.tensor(np.random.default_rng(1).normal(size=(b.n, 3)), device="cuda")
    xb, ub, tb = AD.eval_vjp(b, abar)
    res["batch_xb"], res["batch_tb"] = xb.cpu().numpy(), tb.cpu().numpy()
    b.close()
    np.savez(out_path, **res)


def test_debug_build_matches_release_bitwise(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10134_gb300 import _build
    _build.build(debug=True)
    dbg = tmp_path / "debug.npz"
    env = dict(os.environ, MDPD_DEBUG="1", PYTHONPATH=ROOT + os.pathsep + HERE)
    code = ("import sys; sys.path[:0] = [%r, %r]; import test_gpu_debug_build as T; "
            "from paper_1903_10134_gb300 import mdpd; assert mdpd.debug_build(); "
            "T.run_cases(%r); print('debug', mdpd.library_path())" % (ROOT, HERE, str(dbg)))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "libmdpd_gb300_debug.so" in r.stdout
    rel = tmp_path / "release.npz"
    run_cases(rel)
    a, b = np.load(dbg), np.load(rel)
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
