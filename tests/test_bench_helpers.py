"""Host logic of bench.py: the candidate-test count behind the density pass's
roofline figure, checked against a direct count over cells."""
import importlib.util
import math
import os

import numpy as np
import pytest

from paper_1903_10134_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("periodic", [(1, 1, 1), (1, 0, 1), (0, 0, 0)])
def test_candidate_count_matches_direct_count(periodic):
    B = _bench()
    rng = np.random.default_rng(3)
    p = I.MDPDParams(box_lo=(-1.0, 0.5, 2.0), box=(5.3, 4.1, 6.7), periodic=periodic)
    n = 400
    x = np.array(p.box_lo) + rng.random((n, 3)) * np.array(p.box)
    nc = [max(1, int(math.floor(p.box[k] / p.rc))) for k in range(3)]
    got = B.candidate_tests(x, p, nc)
    h = np.array(p.box) / nc
    q = np.clip(np.floor((x - np.array(p.box_lo)) / h).astype(int), 0, np.array(nc) - 1)
    want = 0
    for i in range(n):
        for j in range(n):
            ok = True
            for k in range(3):
                d = q[j, k] - q[i, k]
                if periodic[k]:
                    d = (d + 1) % nc[k] - 1
                if d not in (-1, 0, 1):
                    ok = False
            want += ok
    assert got == want


def test_split_candidate_count_matches_direct_count():
    """With frozen particles (the split density pass) only mobile homes scan
    their neighbourhood; frozen homes take no candidate tests."""
    B = _bench()
    rng = np.random.default_rng(5)
    p = I.MDPDParams(box=(5.0, 4.2, 6.1), periodic=(1, 1, 0))
    n = 300
    x = rng.random((n, 3)) * np.array(p.box)
    frozen = rng.random(n) < 0.4
    nc = [max(1, int(math.floor(p.box[k] / p.rc))) for k in range(3)]
    got = B.candidate_tests(x, p, nc, frozen)
    h = np.array(p.box) / nc
    q = np.clip(np.floor(x / h).astype(int), 0, np.array(nc) - 1)
    want = 0
    for i in range(n):
        for j in range(n):
            if frozen[i]:
                continue
            ok = True
            for k in range(3):
                d = q[j, k] - q[i, k]
                if p.periodic[k]:
                    d = (d + 1) % nc[k] - 1
                if d not in (-1, 0, 1):
                    ok = False
            want += ok
    assert got == want
    assert got < B.candidate_tests(x, p, nc)
