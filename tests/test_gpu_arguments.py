"""Argument checks of the entry points beyond the base path: every bad
pointer, size, control or option is refused with OCP_ERR_INVALID_ARG before
anything is launched, and a refused call leaves the grid usable; a bad
well control found on the device sets the sticky status."""
import numpy as np
import pytest

from _gpu_common import dev_state, need_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup():
    need_gpu()
    from paper_2406_10862_gb300 import ocp as O
    from paper_2406_10862_gb300 import workloads as W
    g, s = W.tiny(5, 4, 3, seed=61)
    return O, O.load(), g, s, O.Grid(g)


def test_null_and_bad_arguments_are_refused():
    O, lib, g, s, grid = _setup()
    INV = O.OCP_ERR_INVALID_ARG
    h = grid._h
    un, fn, uo, fo = dev_state(s)
    p = un.data_ptr()
    # wells as unknowns
    assert lib.ocp_linearize_wells(h, p, fn.data_ptr(), uo.data_ptr(), fo.data_ptr(), 1.0, None, None, None, None,
                                   None, None, None, None, None, None) == INV
    assert lib.ocp_linearize_wells(h, p, fn.data_ptr(), uo.data_ptr(), fo.data_ptr(), 0.0, None, None, None, None,
                                   None, None, None, None, None, None) == INV
    assert lib.ocp_bicgstab_wells(h, None, None, None, None, None, None, None, None, 1e-8, 10, 0, None, None, None,
                                  None) == INV
    work = grid.solver_work()
    assert lib.ocp_bicgstab_wells(h, p, None, None, None, p, None, p, None, 1e-8, 10, 0, work.data_ptr(), None,
                                  None, None) == INV                       # b == x
    assert lib.ocp_well_update(h, None, None, 1.0, None, None, None, None) == INV
    assert lib.ocp_residual_norms(h, None, 1.0, None, None, None, None) == INV
    # (P, N)
    assert lib.ocp_linearize_pn(h, None, None, 1.0, None, None, None, None, None, None, None) == INV
    assert lib.ocp_pn_update(h, None, None, 1.0, None, None, None) == INV
    assert lib.ocp_pn_norms(h, None, 1.0, None, None) == INV
    assert lib.ocp_pn_from_natural(h, None, None, None, None) == INV
    # IMPEC
    assert lib.ocp_impec_pressure(h, p, -1.0, p, p, None) == INV
    assert lib.ocp_impec_update(h, p, p, 1.0, p, None) == INV              # pn_old == pn_new
    assert lib.ocp_bicgstab_scalar(h, p, p, p, 1e-8, 10, work.data_ptr(), None, None, None) == INV
    # coupling: subdomain counts outside [1, cells per direction], bad threshold
    lab = torch.empty(64, dtype=torch.int32, device="cuda")
    wk = torch.empty(256, dtype=torch.int32, device="cuda")
    for px, py, pz, thr in ((0, 1, 1, 0.1), (6, 1, 1, 0.1), (1, 5, 1, 0.1), (1, 1, 4, 0.1), (1, 1, 1, -1.0),
                            (1, 1, 1, float("nan"))):
        assert lib.ocp_coupling_components(h, p, fn.data_ptr(), uo.data_ptr(), fo.data_ptr(), thr, px, py, pz,
                                           lab.data_ptr(), wk.data_ptr(), None) == INV
    assert lib.ocp_coupling_work_ints(0, 1, 1) == 0
    # the grid still works after the refusals
    r, v, _ = grid.linearize(un, fn, uo, fo, s.dt)
    assert grid.status() == 0


def test_bad_well_control_sets_the_sticky_status():
    O, lib, g, s, grid = _setup()
    un, fn, uo, fo = dev_state(s)
    p = torch.as_tensor(np.array([4000.0, 5200.0]), device="cuda")
    # rate control of a phase the two-phase-or-three-phase model has no index for
    c = O.well_controls([(1, 7, 100.0), (0, 2, 5200.0)], [1000.0, 8000.0], grid.device)
    grid.linearize_wells(un, fn, uo, fo, s.dt, p, c)
    assert grid.status() == O.OCP_ERR_INVALID_ARG
    assert grid.status() == 0                   # reading the status clears it
    c = O.well_controls([(3, 1, 100.0), (0, 2, 5200.0)], [1000.0, 8000.0], grid.device)   # unknown mode
    grid.linearize_wells(un, fn, uo, fo, s.dt, p, c)
    assert grid.status() == O.OCP_ERR_INVALID_ARG
    # a valid control afterwards is clean
    c = O.well_controls([(1, 1, 100.0), (0, 2, 5200.0)], [1000.0, 8000.0], grid.device)
    grid.linearize_wells(un, fn, uo, fo, s.dt, p, c)
    assert grid.status() == 0
