"""The C-ABI library on the CPU: it builds, loads, exports every entry point
declared in include/pt.h, and its host-only calls (basis listing, workspace
size, parameter checks) agree with the oracle. No device work is done here.
"""
import os
import re

import numpy as np
import pytest

import synthetic as syn
from oracle.discretization import Grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_1905_01348_gb300 as p
    from paper_1905_01348_gb300 import build as b
    if not os.path.exists(p._native.LIB_PATH):
        b.build()
    p.load()
    return p


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pt.h")).read()
    return sorted(set(re.findall(r"\b(pt_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(pkg):
    import ctypes
    lib = ctypes.CDLL(pkg._native.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("name,over", [
    ("si8", {}),
    ("si8", dict(n=(32, 24, 48), cell=(10.26, 8.1, 15.0))),
    ("si64", {}),
])
def test_basis_matches_oracle(pkg, name, over):
    w = syn.si_workload(name, **over)
    p = pkg.make_params(w)
    g = Grid(w["n"], w["cell"], w["ecut"])
    assert pkg.pt_basis_size(p) == g.npw
    assert np.array_equal(pkg.pt_basis_indices(p), g.basis)


def test_workspace_and_parameter_checks(pkg):
    w = syn.si_workload("si8")
    p = pkg.make_params(w)
    b64 = pkg.pt_workspace_size(p)
    bmix = pkg.pt_workspace_size(pkg.make_params(dict(w, precision="mixed")))
    assert b64 > bmix > 0
    bad = pkg.make_params(dict(w, n=(30, 32, 32)))
    with pytest.raises(pkg.PtError):
        pkg.pt_workspace_size(bad)
    bad = pkg.make_params(dict(w, anderson_dim=25))
    with pytest.raises(pkg.PtError):
        pkg.pt_workspace_size(bad)
    assert "grid" in pkg.pt_last_error(None) or "anderson" in pkg.pt_last_error(None)


def test_null_handle_calls_fail_with_a_message(pkg):
    """Entry points given a NULL handle or output return PT_ERR_INVALID without touching the
    device and leave a message naming the call in pt_last_error(NULL)."""
    import ctypes
    lib = ctypes.CDLL(pkg._native.LIB_PATH)
    lib.pt_last_error.restype = ctypes.c_char_p
    lib.pt_last_error.argtypes = [ctypes.c_void_p]
    vp = ctypes.c_void_p
    calls = {
        "pt_build_ace": (),
        "pt_apply_h": (vp(1), vp(1), 1, 0),
        "pt_exchange": (vp(1),),
        "pt_cn_step": (None,),
        "pt_rk4_step": (None,),
        "pt_propagate": (1, None),
        "pt_get_orbitals": (vp(1),),
        "pt_set_orbitals": (vp(1),),
        "pt_get_state": (vp(1), vp(1), None),
        "pt_set_state": (vp(1), vp(1), ctypes.c_int64(0)),
        "pt_observables": (None, None),
        "pt_orbitals_device": (vp(1),),
        "pt_set_timing": (1,),
        "pt_get_timing": (None, None, None, 0),
    }
    for name, args in calls.items():
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        assert fn(None, *args) == 1, name
        assert lib.pt_last_error(None).decode().startswith(name + ":"), name
    lib.pt_launch_count.restype = ctypes.c_int
    assert lib.pt_launch_count(None) == 1
    assert lib.pt_last_error(None).decode().startswith("pt_launch_count:")
    assert lib.pt_destroy(None) == 0
