"""GPU parity of the (P, N) path with the volume balance (Sec. 2.1, eq. 4):
the phase split, the reduced system after the elimination of the volume rows,
the full system, the update with N_w recovered, and a Newton step, each
against the oracle on the same seeded inputs."""
import numpy as np
import pytest

from _gpu_common import RTOL_J, RTOL_R, assert_scaled_close, need_gpu
from oracle.pn import eliminate_volume_row, linearize_pn, natural_to_pn, newton_step_pn
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _state(nx, ny, nz, nphase, seed, off=1.0, dt=2.5):
    g, s = W.tiny(nx, ny, nz, nphase=nphase, seed=seed, frac_unsat=0.35 if nphase == 3 else 0.0, rs_hi=0.7)
    x_new = natural_to_pn(g, s.u_new, s.flag_new)
    x_new[1] *= off                      # off = 1: on the volume-balance manifold
    x_old = natural_to_pn(g, s.u_old, s.flag_old)
    return g, x_new, x_old, dt


CASES = [(5, 4, 3, 3, 3, 1.0), (5, 4, 3, 3, 3, 1.002), (7, 5, 4, 3, 11, 0.997), (6, 5, 3, 2, 4, 1.0),
         (6, 5, 3, 2, 12, 1.003), (17, 9, 6, 3, 13, 1.001)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%dx%d-np%d-s%d-off%g" % c)
def test_linearize_pn_matches_oracle(case):
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    nx, ny, nz, nphase, seed, off = case
    g, x_new, x_old, dt = _state(nx, ny, nz, nphase, seed, off)
    full = linearize_pn(g, x_new, x_old, dt)
    red = eliminate_volume_row(g, full)
    grid = ocp.Grid(g)
    o = grid.linearize_pn(_T(x_new.ravel()), _T(x_old.ravel()), dt, full=True)
    assert grid.status() == 0
    N, nb = g.N, nphase
    assert np.array_equal(o["flag"].cpu().numpy()[:N] if nb == 3 else np.zeros(N, np.int8),
                          full["flag"] if nb == 3 else np.zeros(N, np.int8))
    assert_scaled_close(o["residual"].cpu().numpy(), red["R"], red["R_mag"], RTOL_R, "reduced residual")
    assert_scaled_close(o["bsr_val"].cpu().numpy(), red["val"], red["val_mag"], RTOL_J, "reduced bsr_val")
    assert_scaled_close(o["residual_full"].cpu().numpy(), full["R"], full["R_mag"], RTOL_R, "full residual")
    assert_scaled_close(o["bsr_val_full"].cpu().numpy(), full["val"], full["val_mag"], RTOL_J, "full bsr_val")
    elim = o["elim"].cpu().numpy().reshape(nb + 1, N)
    ref = np.stack([red["c"][:, 0]] + [red["c"][:, k] for k in range(2, nb + 1)] + [red["c_r"]])
    assert np.allclose(elim, ref, rtol=1e-12, atol=1e-15 * np.abs(ref).max())


def test_pn_update_recovers_nw():
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    g, x_new, x_old, dt = _state(5, 4, 3, 3, 3, 1.002)
    grid = ocp.Grid(g)
    o = grid.linearize_pn(_T(x_new.ravel()), _T(x_old.ravel()), dt)
    rng = np.random.default_rng(2)
    dx = rng.normal(size=3 * g.N) * np.tile([10.0, 1e-3, 1e-3], g.N)
    pn = _T(x_new.ravel()).clone()
    dmax = grid.empty(4)
    grid.pn_update(pn, _T(dx), -1.0, o["elim"], dmax)
    elim = o["elim"].cpu().numpy().reshape(4, g.N)
    x = dx.reshape(-1, 3)
    xw = elim[3] - elim[0] * x[:, 0] - elim[1] * x[:, 1] - elim[2] * x[:, 2]
    ref = x_new - np.stack([x[:, 0], xw, x[:, 1], x[:, 2]])
    got = pn.cpu().numpy().reshape(4, g.N)
    assert np.allclose(got, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max(axis=1, keepdims=True))
    full = np.stack([x[:, 0], xw, x[:, 1], x[:, 2]])
    assert np.allclose(dmax.cpu().numpy(), np.abs(full).max(axis=1), rtol=1e-14)


@pytest.mark.parametrize("nphase", [2, 3])
def test_newton_step_pn_matches_oracle(nphase):
    need_gpu()
    from paper_2406_10862_gb300 import fim, ocp
    g, s = W.tiny(6, 5, 3, nphase=nphase, seed=4, frac_unsat=0.3 if nphase == 3 else 0.0, rs_hi=0.7)
    x_old = natural_to_pn(g, s.u_old, s.flag_old)
    ref, flag_ref, it_ref = newton_step_pn(g, x_old, 1.0)
    grid = ocp.Grid(g)
    st = fim.Stepper(grid)
    pn, flag, it = st.step_pn(_T(x_old.ravel()), 1.0)
    got = pn.cpu().numpy().reshape(nphase + 1, g.N)
    if nphase == 3:
        assert np.array_equal(flag.cpu().numpy(), flag_ref)
    assert np.allclose(got[0], ref[0], rtol=0, atol=1e-7)
    for e in range(1, nphase + 1):
        assert np.allclose(got[e], ref[e], rtol=1e-10, atol=1e-14)
    assert abs(it - it_ref) <= 1


@pytest.mark.parametrize("nphase", [2, 3])
def test_pn_from_natural_matches_oracle(nphase):
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    g, s = W.tiny(7, 6, 4, nphase=nphase, seed=14, frac_unsat=0.3 if nphase == 3 else 0.0, rs_hi=0.7)
    grid = ocp.Grid(g)
    got = grid.pn_from_natural(_T(s.u_new.ravel()), _T(s.flag_new)).cpu().numpy().reshape(nphase + 1, g.N)
    ref = natural_to_pn(g, s.u_new, s.flag_new)
    assert np.allclose(got, ref, rtol=1e-14, atol=0.0)


@pytest.mark.parametrize("nphase", [3, 2])
def test_linearize_pn_is_the_same_for_every_launch_shape(nphase):
    """The (P, N) path leaves the accumulation out of the cell stage; every
    launch shape, the one-cluster launch included, gives the same bits."""
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    g, x_new, x_old, dt = _state(7, 5, 4, nphase, 11, 1.001)
    grid = ocp.Grid(g)
    shapes = [dict(cells_per_tile=[128, 128, 256], ctas_per_sm=[0, 0, 0], ordered=0),
              dict(cells_per_tile=[64, 64, 256], ctas_per_sm=[0, 0, 0], ordered=2),
              dict(cells_per_tile=[32, 32, 32], ctas_per_sm=[0, 0, 0], ordered=3),
              dict(cells_per_tile=[32, 32, 32], ctas_per_sm=[0, 0, 0], ordered=4)]
    ref = None
    for sh in shapes:
        grid.set_shape(sh)
        o = grid.linearize_pn(_T(x_new.ravel()), _T(x_old.ravel()), dt, full=True)
        assert grid.status() == 0, sh
        got = {k: v.clone() for k, v in o.items()}
        if ref is None:
            ref = got
            continue
        for k in ref:
            a, b = got[k], ref[k]
            if a.dtype == torch.float64:
                a, b = a.view(torch.int64), b.view(torch.int64)
            assert torch.equal(a, b), (sh, k)
