"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, exports
every entry point that include/mdpd.h declares, and validates arguments on
the host before touching a GPU."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1903_10134_gb300 import _build, inputs as I, mdpd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mdpd_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return mdpd.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mdpd_create", "mdpd_set_walls", "mdpd_step", "mdpd_get_state",
                     "mdpd_forces", "mdpd_destroy", "mdpd_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(mdpd_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)
    assert set(mdpd.SYMBOLS) <= set(declared_functions())


def test_params_struct_layout():
    # mdpd_params: 3+3 doubles, 4 int32, 4 doubles, 3*64 doubles, 3 doubles, 4 x 32-bit
    assert C.sizeof(mdpd.Params) == 8 * 6 + 4 * 4 + 8 * 4 + 8 * 192 + 8 * 3 + 4 * 4


def test_library_targets_sm103a():
    out = subprocess.run(["cuobjdump", "--list-elf", _build.LIB], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def _bad(params=None, n=10, **over):
    w = I.tiny(n, (4.0, 4.0, 4.0), 1)
    p = params or w.params
    for k, v in over.items():
        setattr(p, k, v)
    with pytest.raises(mdpd.MDPDError) as e:
        mdpd.mdpd_create(p, w.pos, w.vel, w.type, 1)
    return e.value


@pytest.mark.parametrize("field,value", [
    ("ntypes", 0), ("ntypes", 9), ("rc", 0.0), ("rd", 1.5), ("dt", -0.01),
    ("precision", 3), ("xi_dist", 2), ("box", (2.0, 4.0, 4.0)),
])
def test_invalid_params_rejected_on_host(field, value):
    err = _bad(**{field: value})
    assert err.name == "INVALID_ARG"


def test_asymmetric_table_rejected():
    p = I.MDPDParams(ntypes=2)
    p.A[0, 1] = -30.0
    err = _bad(params=p)
    assert err.name == "INVALID_ARG" and "symmetric" in str(err)


def test_type_out_of_range_rejected():
    w = I.tiny(10, (4.0, 4.0, 4.0), 1)
    t = w.type.copy()
    t[3] = 5
    with pytest.raises(mdpd.MDPDError) as e:
        mdpd.mdpd_create(w.params, w.pos, w.vel, t, 1)
    assert e.value.name == "INVALID_ARG"


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.mdpd_step(None, 1) == -1
    assert lib.mdpd_sync(None) == -1
    assert lib.mdpd_get_state(None, None, None, None, None) == -1
    lib.mdpd_destroy(None)


def test_debug_library_builds_and_exports_every_declared_symbol():
    """The index-checking build (-DMDPD_DEBUG, libmdpd_gb300_debug.so)
    compiles for sm_103a and exports the same entry points."""
    path = _build.build(debug=True)
    assert path == _build.LIB_DEBUG and os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(mdpd_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
