"""GPU parity of the wells as unknowns (Sec. 3.4.1 "w" rows and columns,
Sec. 3.2.4 pressure monitoring): the linearisation with bottom-hole
pressures and controls, the Schur-complement solve, the well update with its
pressure-limit switch, the residual norms, and the Newton loop with rate
controls, each against the oracle on the same seeded inputs."""
import numpy as np
import pytest

from _gpu_common import RTOL_J, RTOL_R, assert_scaled_close, dev_state, need_gpu
from oracle.linearize import linearize
from oracle.newton import full_system, newton_step_wells, residual_norms
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _grid(g):
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    return ocp, ocp.Grid(g)


def _T(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype)


CASES = [
    # (nx, ny, nz, nphase, seed, p_bh, controls)
    (6, 5, 3, 3, 4, [4300.0, 5300.0], [(1, 1, 150.0), (1, 2, 400.0)]),
    (6, 5, 3, 3, 5, [4300.0, 5300.0], [(0, 1, 4350.0), (1, 2, 400.0)]),
    (7, 4, 4, 2, 6, [4400.0, 5200.0], [(1, 1, 100.0), (1, 0, 300.0)]),
    (9, 7, 5, 3, 7, [3900.0, 5600.0], [(1, 0, 10.0), (0, 2, 5500.0)]),   # producer on its water rate
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%dx%d-np%d-s%d" % c[:5])
def test_linearize_wells_matches_oracle(case):
    nx, ny, nz, nphase, seed, p, ctrl = case
    g, s = W.tiny(nx, ny, nz, nphase=nphase, seed=seed, frac_unsat=0.3 if nphase == 3 else 0.0)
    ocp, grid = _grid(g)
    ref = linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt, p_bh=np.array(p), controls=ctrl)
    un, fn, uo, fo = dev_state(s)
    c = ocp.well_controls(ctrl, [0.0, 1e9], grid.device)
    out = grid.linearize_wells(un, fn, uo, fo, s.dt, _T(p), c)
    assert grid.status() == 0
    nb = g.nphase
    assert_scaled_close(out["residual"].cpu().numpy(), ref["R"], ref["R_mag"], RTOL_R, "residual")
    assert_scaled_close(out["bsr_val"].cpu().numpy(), ref["val"], ref["val_mag"], RTOL_J, "bsr_val")
    assert_scaled_close(out["well_res"].cpu().numpy(), ref["well_res"], ref["well_res_mag"], RTOL_R, "well_res")
    assert_scaled_close(out["well_d"].cpu().numpy(), ref["well_D"], ref["well_D_mag"], RTOL_J, "well_d")
    npf = grid.nperf
    assert_scaled_close(out["well_b"].cpu().numpy()[:npf * nb], ref["well_B"], ref["well_B_mag"], RTOL_J, "well_b")
    assert_scaled_close(out["well_c"].cpu().numpy()[:npf * nb], ref["well_C"], ref["well_C_mag"], RTOL_J, "well_c")


def test_pressure_controls_reproduce_fixed_pressure_wells_bitwise():
    g, s = W.tiny(6, 5, 3, seed=8, frac_unsat=0.3)
    ocp, grid = _grid(g)
    un, fn, uo, fo = dev_state(s)
    r0, v0, _ = grid.linearize(un, fn, uo, fo, s.dt)
    p = [w.p_bh for w in g.wells]
    c = ocp.well_controls([(0, 1, q) for q in p], [0.0, 1e9], grid.device)
    out = grid.linearize_wells(un, fn, uo, fo, s.dt, _T(p), c)
    assert torch.equal(out["residual"], r0) and torch.equal(out["bsr_val"], v0)
    assert torch.all(out["well_res"][:2] == 0) and torch.all(out["well_d"][:2] == 1)


@pytest.mark.parametrize("transpose", [False, True])
def test_schur_solve_matches_direct_solve(transpose):
    # the oracle's own Jacobian with well terms, solved by the library's
    # Schur-complement BiCGSTAB and by a sparse direct solve
    import scipy.sparse.linalg as spla
    g, s = W.tiny(6, 5, 3, seed=4, frac_unsat=0.3)
    p = np.array([4300.0, 5300.0])
    ctrl = [(1, 1, 150.0), (1, 2, 400.0)]
    o = linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt, p_bh=p, controls=ctrl)
    ocp, grid = _grid(g)
    rng = np.random.default_rng(3)
    nb, N = g.nphase, g.N
    b = rng.normal(size=N * nb)
    bw = rng.normal(size=2)
    A = full_system(g, o)
    if transpose:
        A = A.T.tocsc()
    ref = spla.spsolve(A, np.concatenate([b, bw]))
    x, xw = torch.zeros(N * nb, dtype=torch.float64, device="cuda"), torch.zeros(2, dtype=torch.float64, device="cuda")
    st, it, rr = grid.bicgstab_wells(_T(o["val"].ravel()), _T(o["well_B"].ravel()), _T(o["well_C"].ravel()),
                                     _T(o["well_D"]), _T(b), _T(bw), x, xw, 1e-13, 2000, transpose=transpose)
    assert st == 0
    got = np.concatenate([x.cpu().numpy(), xw.cpu().numpy()])
    # the full system's residual, and the solution against the direct one
    res = A @ got - np.concatenate([b, bw])
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(np.concatenate([b, bw])) * 1e3
    assert np.allclose(got, ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max())


def test_residual_norms_match_oracle():
    g, s = W.tiny(6, 5, 3, seed=9, frac_unsat=0.3)
    p = np.array([4300.0, 5300.0])
    ctrl = [(1, 1, 150.0), (0, 2, 5300.5)]
    o = linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt, p_bh=p, controls=ctrl)
    cnv, wr = residual_norms(g, o, s.dt, ctrl)
    ocp, grid = _grid(g)
    c = ocp.well_controls(ctrl, [0.0, 1e9], grid.device)
    nrm = grid.residual_norms(_T(o["R"].ravel()), s.dt, _T(o["well_res"]), c).cpu().numpy()
    assert np.allclose(nrm[:3], cnv, rtol=1e-15, atol=0.0)
    assert nrm[3] == pytest.approx(wr, rel=1e-15)


def test_well_update_switches_at_the_limit():
    g, s = W.tiny(6, 5, 3, seed=4, frac_unsat=0.3)
    ocp, grid = _grid(g)
    # producer (well 0) rate-controlled, limit 4000; injector rate-controlled, limit 6000
    c = ocp.well_controls([(1, 1, 150.0), (1, 2, 400.0)], [4000.0, 6000.0], grid.device)
    p = _T([4100.0, 5900.0])
    dpmax = grid.empty(1)
    nsw = torch.zeros(1, dtype=torch.int32, device="cuda")
    grid.well_update(p, _T([50.0, -20.0]), -1.0, c, dpmax, nsw)      # 4050, 5920: no switch
    assert p.cpu().tolist() == [4050.0, 5920.0] and int(nsw.item()) == 0 and dpmax.item() == 50.0
    grid.well_update(p, _T([100.0, -100.0]), -1.0, c, dpmax, nsw)    # 3950 < 4000, 6020 > 6000
    assert p.cpu().tolist() == [4000.0, 6000.0] and int(nsw.item()) == 2
    assert ocp.read_controls(c) == [(0, 1, 4000.0, 4000.0), (0, 2, 6000.0, 6000.0)]


@pytest.mark.parametrize("nphase", [2, 3])
def test_newton_with_rate_controls_matches_oracle(nphase):
    from paper_2406_10862_gb300 import fim
    g, s = W.tiny(6, 5, 3, nphase=nphase, seed=4, frac_unsat=0.3 if nphase == 3 else 0.0)
    ctrl = [(1, 1, 200.0), (1, 2 if nphase == 3 else 0, 500.0)]
    lim = [1000.0, 8000.0]
    p0 = [3000.0, 6000.0]
    u_ref, f_ref, p_ref, c_ref, o_ref, it_ref = newton_step_wells(g, s.u_old, s.flag_old, 1.0, np.array(p0),
                                                                  ctrl, lim)
    ocp, grid = _grid(g)
    st = fim.Stepper(grid)
    c = ocp.well_controls(ctrl, lim, grid.device)
    u, f, p, it = st.step_wells(_T(s.u_old.ravel()), _T(s.flag_old), 1.0, _T(p0), c)
    assert np.array_equal(f.cpu().numpy(), f_ref)
    assert np.allclose(u.cpu().numpy().reshape(nphase, -1), u_ref, rtol=1e-8, atol=1e-9)
    assert np.allclose(p.cpu().numpy(), p_ref, rtol=1e-10)
    assert abs(it - it_ref) <= 1
    assert [r[:3] for r in ocp.read_controls(c)] == [tuple(x) for x in c_ref]


def test_newton_pressure_limit_switch_matches_oracle():
    from paper_2406_10862_gb300 import fim
    g, s = W.tiny(6, 5, 3, seed=4, frac_unsat=0.3)
    ctrl = [(1, 1, 1e6), (0, 2, 5100.0)]
    lim = [4000.0, 8000.0]
    p0 = [4500.0, 5100.0]
    u_ref, f_ref, p_ref, c_ref, o_ref, it_ref = newton_step_wells(g, s.u_old, s.flag_old, 1.0, np.array(p0),
                                                                  ctrl, lim)
    ocp, grid = _grid(g)
    st = fim.Stepper(grid)
    c = ocp.well_controls(ctrl, lim, grid.device)
    u, f, p, it = st.step_wells(_T(s.u_old.ravel()), _T(s.flag_old), 1.0, _T(p0), c)
    assert ocp.read_controls(c)[0][:3] == (0, 1, 4000.0) and c_ref[0] == (0, 1, 4000.0)
    assert p.cpu().tolist()[0] == 4000.0
    assert np.allclose(u.cpu().numpy().reshape(3, -1), u_ref, rtol=1e-8, atol=1e-9)


SHAPES = [dict(cells_per_tile=[128, 128, 256], ctas_per_sm=[0, 0, 0], ordered=0),
          dict(cells_per_tile=[64, 64, 256], ctas_per_sm=[0, 0, 0], ordered=2),
          dict(cells_per_tile=[32, 32, 32], ctas_per_sm=[0, 0, 0], ordered=3),
          dict(cells_per_tile=[32, 32, 32], ctas_per_sm=[0, 0, 0], ordered=4)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%dx%d-np%d-s%d" % c[:5])
def test_linearize_wells_is_the_same_for_every_launch_shape(case):
    """The well terms with bottom-hole pressures as unknowns go through the
    cell stage of every launch shape, including the one-cluster launch that
    splits a perforated cell's terms over warps: the same bits everywhere."""
    nx, ny, nz, nphase, seed, p, ctrl = case
    g, s = W.tiny(nx, ny, nz, nphase=nphase, seed=seed, frac_unsat=0.3 if nphase == 3 else 0.0)
    ocp, grid = _grid(g)
    un, fn, uo, fo = dev_state(s)
    c = ocp.well_controls(ctrl, [0.0, 1e9], grid.device)
    ref = None
    for sh in SHAPES:
        grid.set_shape(sh)
        out = grid.linearize_wells(un, fn, uo, fo, s.dt, _T(p), c)
        assert grid.status() == 0, sh
        npf = grid.nperf * g.nphase
        got = {k: (v[:npf] if k in ("well_b", "well_c") else v).clone() for k, v in out.items()
               if isinstance(v, torch.Tensor)}
        if ref is None:
            ref = got
            continue
        for k in ref:
            assert torch.equal(got[k].view(torch.int64), ref[k].view(torch.int64)), (sh, k)
