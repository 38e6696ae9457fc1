"""The C library builds here (no GPU needed), exports every entry point its
headers declare, and rejects malformed descriptors before touching CUDA."""
import copy
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2406_10862_gb300 import build as B
from paper_2406_10862_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2406_10862_gb300 import ocp as O
    return O.load()


def declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^\s*(?:ocp_status|const char\*|int64_t|int|void)\s+(ocp_\w+)\s*\(", src, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert "ocp_linearize" in names and "ocp_adjoint_vjp" in names and "ocp_bsr_spmv" in names
    for n in names:
        assert hasattr(lib, n), n
    from paper_2406_10862_gb300 import ocp as O
    assert set(O.EXPORTS) <= names


def test_library_targets_sm103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _create(lib, g):
    from paper_2406_10862_gb300 import ocp as O
    d, keep = O.make_desc(g)
    h = ctypes.c_void_p()
    st = lib.ocp_grid_create(ctypes.byref(d), 0, ctypes.byref(h))
    return st, lib.ocp_last_error().decode()


BAD = [
    ("nphase", 4, "nphase"),
    ("nx", 0, "nx"),
    ("dz", -1.0, "dz"),
    ("tab_p", np.r_[W.synthetic_tables()["tab_p"][:-1], 0.0], "tab_p"),
    ("tab_Rs", np.r_[W.synthetic_tables()["tab_Rs"][:-1], 0.0], "tab_Rs"),
    ("tab_Bo", -W.synthetic_tables()["tab_Bo"], "tab_Bo"),
    ("nw", 0.5, "exponent"),
    ("swc", 0.9, "swc"),
    ("kro_cw", 0.0, "kro_cw"),
]


@pytest.mark.parametrize("field,value,msg", BAD)
def test_bad_descriptor_is_rejected_on_the_host(lib, field, value, msg):
    g, _ = W.tiny(3, 2, 2, seed=1)
    setattr(g, field, value)
    st, err = _create(lib, g)
    assert st == 1 and msg.split()[0].lower() in err.lower(), err


def test_bad_cell_data_and_wells_are_rejected(lib):
    g, _ = W.tiny(3, 2, 2, seed=1)
    h = copy.deepcopy(g)
    h.phi[3] = 0.0
    assert _create(lib, h)[0] == 1
    h = copy.deepcopy(g)
    h.lnk[2] = np.nan
    assert _create(lib, h)[0] == 1
    h = copy.deepcopy(g)
    h.wells[0].cells = np.array([h.N])
    st, err = _create(lib, h)
    assert st == 1 and "range" in err
    h = copy.deepcopy(g)
    h.wells[1].cells = h.wells[0].cells.copy()
    st, err = _create(lib, h)
    assert st == 1 and "twice" in err
    h = copy.deepcopy(g)
    h.wells[0].rw = 0.0
    assert _create(lib, h)[0] == 1
    g2, _ = W.tiny(3, 2, 2, nphase=2, seed=1)
    g2.wells[1].phase = 2
    st, err = _create(lib, g2)
    assert st == 1 and "phase" in err


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.ocp_grid_create(None, 0, ctypes.byref(h)) == 1
    assert lib.ocp_linearize(None, None, None, None, None, 1.0, None, None, None, None) == 1
    assert lib.ocp_bsr_spmv(None, None, 1.0, None, 0.0, None, 0, None) == 1
    assert lib.ocp_grid_destroy(None) == 0
