"""ocp_linearize_noalloc against ocp_linearize and the oracle.

The no-allocation entry point serves callers that cannot call cudaMalloc
when they linearise (memory owned by a host framework with its own allocator,
a fixed memory budget).  It must give the same residual, Jacobian and
face fluxes as the ordinary entry point -- within the tolerances of every
other parity test -- on consecutive calls that reuse its shared scratch, and
reject grids larger than its fixed array.  This file is collected last so a
failure here cannot hide the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

from _gpu_common import RTOL_J, RTOL_R, assert_scaled_close, dev_state, need_gpu, torch
from oracle.linearize import linearize as oracle_linearize
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(O, grid, un, fn, uo, fo, dt, r, v, f):
    lib = O.load()
    return lib.ocp_linearize_noalloc(grid._h, ctypes.c_void_p(un.data_ptr()), ctypes.c_void_p(fn.data_ptr()),
                                     ctypes.c_void_p(uo.data_ptr()), ctypes.c_void_p(fo.data_ptr()), float(dt),
                                     ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                     ctypes.c_void_p(f.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _run_both(O, grid, s):
    un, fn, uo, fo = dev_state(s)
    r0, v0, f0 = grid.linearize(un, fn, uo, fo, s.dt, want_face_flux=True)
    r1 = torch.full_like(r0, float("nan"))
    v1 = torch.full_like(v0, float("nan"))
    f1 = torch.full_like(f0, float("nan"))
    st = _noalloc(O, grid, un, fn, uo, fo, s.dt, r1, v1, f1)
    assert st == 0, O.load().ocp_last_error()
    assert grid.status() == 0
    return [t.cpu().numpy() for t in (r0, v0, f0, r1, v1, f1)]


def _poison_static_scratch(O):
    """Fill most of the shared array with NaN: a 36 000-cell three-phase
    linearisation of a NaN state writes NaN into every scratch field it uses
    (its own grid's status records the non-finite input and is discarded).
    A later call that read an entry it had not written would show it."""
    g, s = W.tiny(40, 30, 30, seed=64, wells=False)
    s.u_new[:] = np.nan
    grid = O.Grid(g)
    un, fn, uo, fo = dev_state(s)
    r = torch.empty(3 * g.N, dtype=torch.float64, device="cuda")
    v = torch.empty(grid.nnzb * 9, dtype=torch.float64, device="cuda")
    f = torch.empty(9 * g.N, dtype=torch.float64, device="cuda")
    assert _noalloc(O, grid, un, fn, uo, fo, s.dt, r, v, f) == 0
    assert grid.status() == O.OCP_ERR_NONFINITE
    assert torch.isnan(r).all()


@pytest.mark.parametrize("nphase,shape", [(3, (12, 9, 5)), (2, (7, 6, 4))])
def test_noalloc_matches_linearize_on_consecutive_calls(nphase, shape):
    need_gpu()
    from paper_2406_10862_gb300 import ocp as O
    g, s1 = W.tiny(*shape, nphase=nphase, seed=61)
    _, s2 = W.tiny(*shape, nphase=nphase, seed=62)     # same grid, a different state
    grid = O.Grid(g)
    _poison_static_scratch(O)
    for s in (s1, s2):
        r0, v0, f0, r1, v1, f1 = _run_both(O, grid, s)
        o = oracle_linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt)
        assert_scaled_close(r1, r0, o["R_mag"], RTOL_R, "noalloc residual")
        assert_scaled_close(v1, v0, o["val_mag"], RTOL_J, "noalloc jacobian")
        assert_scaled_close(f1, f0, o["face_flux_mag"], RTOL_R, "noalloc face flux")
        assert_scaled_close(r1, o["R"], o["R_mag"], RTOL_R, "noalloc residual against the oracle")
        assert_scaled_close(v1, o["val"], o["val_mag"], RTOL_J, "noalloc jacobian against the oracle")


def test_noalloc_rejects_grids_beyond_its_array():
    need_gpu()
    from paper_2406_10862_gb300 import ocp as O
    g, s = W.tiny(60, 50, 14, seed=63)                  # 42 000 cells > 41 943
    grid = O.Grid(g)
    un, fn, uo, fo = dev_state(s)
    r = torch.empty(3 * g.N, dtype=torch.float64, device="cuda")
    v = torch.empty(grid.nnzb * 9, dtype=torch.float64, device="cuda")
    with pytest.raises(O.OcpError) as e:
        grid.linearize_noalloc(un, fn, uo, fo, s.dt, r, v)
    assert e.value.status == O.OCP_ERR_INVALID_ARG and "at most 41943 cells" in str(e.value)
