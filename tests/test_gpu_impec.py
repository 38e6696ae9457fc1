"""GPU parity of one IMPEC step in (P, N): the pressure matrix and right-hand
side, the pressure solve, and the explicit update, against the oracle; and
the update's conservation of every component."""
import numpy as np
import pytest

from _gpu_common import need_gpu
from oracle.impec import impec_step, pressure_system
from oracle.pn import natural_to_pn
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL_A = 1e-12        # matrix entries and right-hand side, relative to their magnitude scales


def _T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


CASES = [(6, 5, 3, 3, 4, 0.5, True), (7, 4, 5, 3, 9, 2.0, True), (6, 5, 3, 2, 4, 1.0, True),
         (9, 6, 4, 3, 15, 0.25, False), (11, 8, 3, 3, 16, 1.0, True)]


def _case(nx, ny, nz, nphase, seed, dt, wells):
    g, s = W.tiny(nx, ny, nz, nphase=nphase, seed=seed, frac_unsat=0.3 if nphase == 3 else 0.0, rs_hi=0.7,
                  wells=wells)
    return g, natural_to_pn(g, s.u_new, s.flag_new), dt


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%dx%d-np%d-s%d-dt%g-w%d" % c)
def test_impec_step_matches_oracle(case):
    need_gpu()
    from paper_2406_10862_gb300 import fim, ocp
    g, x0, dt = _case(*case)
    A, E0, A_mag, E0_mag, _ = pressure_system(g, x0, dt)
    x1, dP, _, _ = impec_step(g, x0, dt)
    grid = ocp.Grid(g)
    rp, ci = grid.pattern()
    rp, ci = rp.cpu().numpy(), ci.cpu().numpy()
    val, rhs = grid.impec_pressure(_T(x0.ravel()), dt)
    assert grid.status() == 0
    rows = np.repeat(np.arange(g.N), np.diff(rp))
    Ad = A.toarray()
    ref = Ad[rows, ci]
    mag = A_mag[rows, ci]
    got = val.cpu().numpy()
    assert np.all(np.abs(got - ref) <= RTOL_A * mag + 1e-300), np.max(np.abs(got - ref) / (mag + 1e-300))
    # every entry of the oracle's matrix lies on the pattern
    assert np.count_nonzero(Ad) == np.count_nonzero(ref)
    assert np.all(np.abs(rhs.cpu().numpy() + E0) <= RTOL_A * E0_mag + 1e-300)
    # the solve
    dp = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    st, it, rr = grid.bicgstab_scalar(val, rhs, dp, 1e-14, 4000)
    assert np.allclose(dp.cpu().numpy(), dP, rtol=1e-8, atol=1e-9 * np.abs(dP).max())
    # the update, from the oracle's own pressure change
    new = grid.impec_update(_T(x0.ravel()), _T(dP), dt).cpu().numpy().reshape(x0.shape)
    assert np.allclose(new[0], x1[0], rtol=0, atol=1e-9)
    for e in range(1, x0.shape[0]):
        scale = np.abs(x1[e] - x0[e]).max() + 1e-300
        assert np.all(np.abs(new[e] - x1[e]) <= 1e-10 * scale + 1e-15 * np.abs(x1[e]))
    # the driver: pressure, solve and update in one call
    pn1, dp1, _ = fim.impec_step(grid, _T(x0.ravel()), dt)
    assert np.allclose(pn1.cpu().numpy().reshape(x0.shape)[0], x1[0], rtol=0, atol=1e-6)


def test_update_conserves_every_component():
    need_gpu()
    from paper_2406_10862_gb300 import fim, ocp
    g, x0, dt = _case(11, 8, 3, 3, 16, 1.0, False)       # no wells: every component is conserved
    grid = ocp.Grid(g)
    pn1, dp, _ = fim.impec_step(grid, _T(x0.ravel()), dt)
    x1 = pn1.cpu().numpy().reshape(x0.shape)
    for e in range(1, 4):
        change = (x1[e] - x0[e]).sum()
        assert abs(change) <= 1e-13 * np.abs(x1[e] - x0[e]).sum() + 1e-15 * np.abs(x0[e]).sum()
