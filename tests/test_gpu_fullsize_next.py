"""Full-size parity of the rows beyond the base path, on the 100x100x20 box
(200 000 cells) in the launch configuration the benchmark times: the (P, N)
linearisation with and without the volume rows eliminated, the IMPEC pressure
system and update, and the linearisation with well unknowns under rate
control.  Sampled rows are recomputed by the oracle on the 3x3x3 window
around each cell (a row depends on nothing outside it); the well rows on the
well's own cells."""
import numpy as np
import pytest

from _gpu_common import RTOL_J, RTOL_R, assert_scaled_close, need_gpu, window
from oracle.dual import D
from oracle.impec import _fluxes_and_sources, pressure_system
from oracle.linearize import linearize
from oracle.pn import eliminate_volume_row, linearize_pn, natural_to_pn
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _sample(g, n, seed):
    rng = np.random.default_rng(seed)
    cells = list(rng.choice(g.N, n, replace=False))
    cells += [0, g.N - 1] + [int(w.cells[0]) for w in g.wells] + [int(w.cells[-1]) for w in g.wells]
    return cells


def test_pn_full_size_sampled():
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    g, s = W.layered_box(frac_unsat=0.2)
    s.u_old[2][s.flag_old == 1] *= 0.7 / 0.9      # keep the undersaturated R_s below saturation
    s.u_new[2][s.flag_new == 1] *= 0.7 / 0.9
    x_new = natural_to_pn(g, s.u_new, s.flag_new)
    x_new[1] *= 1.0005                           # off the volume-balance manifold
    x_old = natural_to_pn(g, s.u_old, s.flag_old)
    dt = 1.0
    grid = ocp.Grid(g)
    o = grid.linearize_pn(_T(x_new.ravel()), _T(x_old.ravel()), dt, full=True)
    assert grid.status() == 0
    rp = grid.pattern()[0].cpu().numpy()
    R3 = o["residual"].cpu().numpy().reshape(-1, 3)
    V3 = o["bsr_val"].cpu().numpy().reshape(-1, 3, 3)
    R4 = o["residual_full"].cpu().numpy().reshape(-1, 4)
    V4 = o["bsr_val_full"].cpu().numpy().reshape(-1, 4, 4)
    for c in _sample(g, 120, 21):
        h, st, centre, cells, _ = window(g, s, c, with_well_index=True)
        full = linearize_pn(h, x_new[:, cells], x_old[:, cells], dt)
        red = eliminate_volume_row(h, full)
        a, b = full["row_ptr"][centre], full["row_ptr"][centre + 1]
        assert_scaled_close(R4[c], full["R"][centre], full["R_mag"][centre], RTOL_R, "full residual %d" % c)
        assert_scaled_close(V4[rp[c]:rp[c + 1]], full["val"][a:b], full["val_mag"][a:b], RTOL_J, "full row %d" % c)
        assert_scaled_close(R3[c], red["R"][centre], red["R_mag"][centre], RTOL_R, "reduced residual %d" % c)
        assert_scaled_close(V3[rp[c]:rp[c + 1]], red["val"][a:b], red["val_mag"][a:b], RTOL_J, "reduced row %d" % c)


def test_impec_full_size_sampled():
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    g, s = W.layered_box()
    x0 = natural_to_pn(g, s.u_new, s.flag_new)
    dt = 0.1
    grid = ocp.Grid(g)
    rp, ci = (t.cpu().numpy() for t in grid.pattern())
    val, rhs = grid.impec_pressure(_T(x0.ravel()), dt)
    val, rhs = val.cpu().numpy(), rhs.cpu().numpy()
    dP = np.random.default_rng(3).normal(0.0, 20.0, g.N)
    x1 = grid.impec_update(_T(x0.ravel()), _T(dP), dt).cpu().numpy().reshape(4, g.N)
    for c in _sample(g, 80, 22):
        h, st, centre, cells, _ = window(g, s, c, with_well_index=True)
        xw = x0[:, cells]
        A, E0, A_mag, E0_mag, old = pressure_system(h, xw, dt)
        row = A.toarray()[centre]
        cols = ci[rp[c]:rp[c + 1]]
        local = {int(x): n for n, x in enumerate(cells)}
        ref = np.array([row[local[int(x)]] for x in cols])
        mag = np.array([A_mag[centre][local[int(x)]] for x in cols])
        assert_scaled_close(val[rp[c]:rp[c + 1]], ref, mag, 1e-12, "pressure row %d" % c)
        assert_scaled_close(rhs[c], -E0[centre], E0_mag[centre], 1e-12, "pressure rhs %d" % c)
        # the explicit update of the centre cell from the same pressure change
        flux, src = _fluxes_and_sources(h, xw, old, D.const(dP[cells], len(cells), 1))
        vdt = g.dx * g.dy * g.dz / 5.614583 / dt
        for e in range(3):
            ref_n = x0[1 + e, c] + (src[e].v[centre] - flux[e].v[centre]) / vdt
            scale = (src[e].m[centre] + flux[e].m[centre]) / vdt
            assert abs(x1[1 + e, c] - ref_n) <= 1e-12 * scale + 1e-15 * abs(ref_n), (c, e)


def test_wells_full_size_rate_controls():
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    g, s = W.layered_box()
    p = np.array([3300.0, 3400.0, 3350.0, 3450.0, 5600.0])
    ctrl = [(1, 1, 2.0e4), (1, 0, 10.0), (1, 1, 3.0e4), (0, 1, 3450.0), (1, 2, 4.0e7)]
    grid = ocp.Grid(g)
    un, fn, uo, fo = (_T(a) for a in (s.u_new.ravel(), s.flag_new, s.u_old.ravel(), s.flag_old))
    c = ocp.well_controls(ctrl, [1000.0] * 4 + [8000.0], grid.device)
    out = grid.linearize_wells(un, fn, uo, fo, s.dt, _T(p), c)
    assert grid.status() == 0
    wres, wd = out["well_res"].cpu().numpy(), out["well_d"].cpu().numpy()
    wb = out["well_b"].cpu().numpy().reshape(-1, 3)
    wc = out["well_c"].cpu().numpy().reshape(-1, 3)
    R = out["residual"].cpu().numpy().reshape(-1, 3)
    k0 = 0
    for iw, w in enumerate(g.wells):
        # the well on its own cells: a grid of the well's column
        cells = np.asarray(w.cells)
        h = W.GridDesc(**{f: getattr(g, f) for f in g.__dataclass_fields__})
        h.nx, h.ny, h.nz = 1, 1, len(cells)
        h.lnk, h.phi = g.lnk[cells], g.phi[cells]
        h.wells = [W.Well(kind=w.kind, phase=w.phase, p_bh=w.p_bh, rw=w.rw, skin=w.skin,
                          cells=np.arange(len(cells), dtype=np.int64))]
        o = linearize(h, s.u_new[:, cells], s.flag_new[cells], s.u_old[:, cells], s.flag_old[cells], s.dt,
                      p_bh=p[iw:iw + 1], controls=[ctrl[iw]])
        n = len(cells)
        assert_scaled_close(wres[iw], o["well_res"][0], o["well_res_mag"][0], RTOL_R, "well %d residual" % iw)
        assert_scaled_close(wd[iw], o["well_D"][0], o["well_D_mag"][0], RTOL_J, "well %d D" % iw)
        assert_scaled_close(wb[k0:k0 + n], o["well_B"], o["well_B_mag"], RTOL_J, "well %d B" % iw)
        assert_scaled_close(wc[k0:k0 + n], o["well_C"], o["well_C_mag"], RTOL_J, "well %d C" % iw)
        k0 += n
        # the perforated cells' rows, on their windows with the unknown p_bh
        for cell in (int(cells[0]), int(cells[len(cells) // 2]), int(cells[-1])):
            hw, st, centre, wcells, kept = window(g, s, cell, with_well_index=True)
            ow = linearize(hw, st.u_new, st.flag_new, st.u_old, st.flag_old, s.dt, p_bh=p[kept],
                           controls=[ctrl[k] for k in kept])
            assert_scaled_close(R[cell], ow["R"][centre], ow["R_mag"][centre], RTOL_R, "perforated row %d" % cell)
