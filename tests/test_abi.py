"""The C-ABI library loads, exports every entry point that include/tlbm.h
declares, and rejects invalid arguments on the host before touching a GPU.
No test here launches device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1511_02155_gb300 as tl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tlbm_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = tl.load_library()
    names = _declared()
    assert "tlbm_create" in names and "tlbm_step" in names and "tlbm_fields" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    lib = tl.load_library()
    for code, name in enumerate(tl.STATUS):
        assert lib.tlbm_status_string(code).decode() == name


def _create(**over):
    lib = tl.load_library()
    a = dict(lattice=9, nx=8, ny=8, nz=1, kappa=(0.01, 0.02, 0.03), alpha=1.0, tau_f=1.0,
             M_phi=0.1, M_psi=0.1, h=(0.0, 0.0, 0.0), prec=1)
    a.update(over)
    h = ctypes.c_void_p()
    k = (ctypes.c_double * 3)(*a["kappa"])
    hh = (ctypes.c_double * 3)(*a["h"])
    rc = lib.tlbm_create(ctypes.byref(h), a["lattice"], a["nx"], a["ny"], a["nz"], k, a["alpha"],
                         a["tau_f"], a["M_phi"], a["M_psi"], hh, None, a["prec"], None)
    return rc, h, lib.tlbm_last_error(None).decode()


@pytest.mark.parametrize("over,status", [
    (dict(lattice=7), 1),
    (dict(nx=0), 1),
    (dict(lattice=9, nz=2), 1),
    (dict(prec=9), 1),
    (dict(kappa=(0.01, -0.02, 0.03)), 2),
    (dict(kappa=(0.01, 0.0, 0.03)), 2),
    (dict(alpha=0.0), 2),
    (dict(tau_f=0.5), 2),
    (dict(M_phi=0.0), 2),
    (dict(M_psi=-1.0), 2),
    (dict(h=(0.0025, 0.0, 0.0)), 2),      # |4h/(alpha kappa)| = 1
    (dict(h=(0.0, 0.0, float("nan"))), 2),
])
def test_create_rejects_invalid_arguments_on_host(over, status):
    rc, h, msg = _create(**over)
    assert rc == status, (rc, msg)
    assert h.value is None
    assert msg


def test_null_handle_calls_return_arg_error():
    lib = tl.load_library()
    out = np.zeros(3)
    assert lib.tlbm_step(None, 1) == 1
    assert lib.tlbm_mass(None, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 1
    assert lib.tlbm_state_bytes(None) == 0
    assert lib.tlbm_launches_per_step(None) == -1
    lib.tlbm_destroy(None)
