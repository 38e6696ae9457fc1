"""GPU parity: the CUDA library through its C interface against the oracle.

Every case feeds the same seeded inputs to ``ocp_linearize`` /
``ocp_bsr_spmv`` / ``ocp_adjoint_vjp`` / ``ocp_well_rates`` and to the CPU
oracle, and compares element by element: the block-CSR pattern bit for bit,
the residual within 1e-12 and the Jacobian within 1e-10 of each entry's
magnitude scale (see ``_gpu_common``).  Sizes run from a single cell up to
the 200 000-cell three-phase box in the configuration the benchmark times;
the 1.12 M-cell oil-water model is checked on sampled rows, each recomputed
by the oracle on the 3x3x3 window around it.
"""
import numpy as np
import pytest

from _gpu_common import (RTOL_J, RTOL_R, RTOL_SPMV, RTOL_VJP, assert_scaled_close, dev_state,
                         gpu_linearize, need_gpu, torch, window)
from oracle.linearize import linearize as oracle_linearize
from oracle.spmv import bsr_spmv as oracle_spmv
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES3 = [(1, 1, 1), (2, 1, 1), (1, 1, 2), (1, 3, 1), (3, 4, 5), (7, 5, 3), (33, 2, 2)]
SHAPES2 = [(1, 1, 1), (4, 3, 2), (5, 1, 7), (17, 9, 2)]


def ocp():
    need_gpu()
    from paper_2406_10862_gb300 import ocp as O
    O.load()
    return O


def orc(g, s, **kw):
    return oracle_linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt, **kw)


def check_linearize(g, s, o=None):
    O = ocp()
    grid = O.Grid(g)
    r, v, ff, st = gpu_linearize(grid, s)
    assert st == 0
    o = o if o is not None else orc(g, s)
    rp, ci = grid.pattern()
    np.testing.assert_array_equal(rp.cpu().numpy(), o["row_ptr"])
    np.testing.assert_array_equal(ci.cpu().numpy(), o["col_idx"])
    assert_scaled_close(r, o["R"], o["R_mag"], RTOL_R, "residual")
    assert_scaled_close(v, o["val"], o["val_mag"], RTOL_J, "jacobian")
    assert_scaled_close(ff, o["face_flux"], o["face_flux_mag"], RTOL_R, "face flux")
    return grid, o, (r, v, ff)


@pytest.mark.parametrize("shape", SHAPES3)
def test_linearize_three_phase(shape):
    g, s = W.tiny(*shape, seed=sum(shape))
    check_linearize(g, s)


@pytest.mark.parametrize("shape", SHAPES2)
def test_linearize_oil_water(shape):
    g, s = W.tiny(*shape, nphase=2, seed=sum(shape) + 100)
    check_linearize(g, s)


def test_linearize_all_undersaturated_and_no_capillarity():
    g, s = W.tiny(4, 3, 3, seed=41, frac_unsat=1.0, pcow_max=0.0, pcgo_max=0.0)
    check_linearize(g, s)


def test_linearize_general_corey_exponents():
    g, s = W.tiny(4, 3, 2, seed=42, nw=3.0, now=1.5, ng=1.0, nog=2.5)
    check_linearize(g, s)


def test_linearize_spe1_shape():
    g, s = W.spe1_like()
    check_linearize(g, s)


def test_linearize_is_deterministic():
    O = ocp()
    g, s = W.tiny(9, 7, 4, seed=43)
    grid = O.Grid(g)
    a = gpu_linearize(grid, s)
    b = gpu_linearize(grid, s)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x.view(np.int64), y.view(np.int64))


@pytest.mark.parametrize("nphase,shape", [(3, (13, 11, 7)), (3, (100, 3, 2)), (2, (9, 30, 5)), (3, (1, 1, 1)),
                                          (3, (40, 40, 3)), (3, (10, 10, 3)), (2, (8, 8, 5)), (3, (16, 8, 4)),
                                          (3, (7, 5, 9))])
def test_launch_shapes_are_bitwise_identical(nphase, shape):
    """Every launch shape of one grid -- tile sizes 32 to 256, one CTA per
    tile or persistent grids, three launches or the ordered launches (face
    stage and assembly in one persistent launch after the cell stage, or
    everything in one), faces and assembly split by direction and equation,
    and for grids of at most 16 tiles of 32 cells the one-cluster launch --
    gives the same bits, and those match the oracle."""
    O = ocp()
    g, s = W.tiny(*shape, nphase=nphase, seed=sum(shape) + 7, frac_unsat=0.3 if nphase == 3 else 0.0)
    grid = O.Grid(g)
    ref = gpu_linearize(grid, s)
    assert ref[3] == 0
    o = orc(g, s)
    assert_scaled_close(ref[0], o["R"], o["R_mag"], RTOL_R, "residual")
    assert_scaled_close(ref[1], o["val"], o["val_mag"], RTOL_J, "jacobian")
    shapes = [dict(cells_per_tile=[128, 128, 256], ctas_per_sm=[0, 0, 0], ordered=0),
              dict(cells_per_tile=[32, 64, 128], ctas_per_sm=[2, 0, 4], ordered=0)]
    for mode in (1, 2):
        for t in (32, 64, 128, 256):
            shapes.append(dict(cells_per_tile=[t, t, 256], ctas_per_sm=[0, 0, 0], ordered=mode))
        shapes.append(dict(cells_per_tile=[64, 128, 256], ctas_per_sm=[0, 1, 0], ordered=mode))
    # face and assembly split by direction and equation
    shapes.append(dict(cells_per_tile=[32, 32, 32], ctas_per_sm=[0, 0, 0], ordered=3))
    shapes.append(dict(cells_per_tile=[128, 32, 32], ctas_per_sm=[2, 1, 3], ordered=3))
    # everything in one thread-block cluster: GB300 runs clusters of 16 CTAs
    tiles = (g.N + 31) // 32
    assert grid.cluster_tiles() == 16
    if tiles <= 16:
        assert grid.get_shape()["ordered"] == 4            # the default for grids that fit
        shapes.append(dict(cells_per_tile=[32, 32, 32], ctas_per_sm=[0, 0, 0], ordered=4))
    else:
        with pytest.raises(O.OcpError):
            grid.set_shape(dict(cells_per_tile=[32, 32, 32], ctas_per_sm=[0, 0, 0], ordered=4))
    for sh in shapes:
        grid.set_shape(sh)
        got = gpu_linearize(grid, s)
        assert got[3] == 0, sh
        for x, y in zip(got[:3], ref[:3]):
            assert np.array_equal(x.view(np.int64), y.view(np.int64)), sh


@pytest.mark.parametrize("nphase", [3, 2])
@pytest.mark.parametrize("alpha,beta,transpose", [(1.0, 0.0, False), (-0.7, 0.3, False), (2.5, 0.0, True),
                                                  (1.0, 1.0, True)])
def test_spmv(nphase, alpha, beta, transpose):
    O = ocp()
    g, s = W.tiny(6, 5, 4, nphase=nphase, seed=44)
    grid, o, (r, v, ff) = check_linearize(g, s)
    rng = np.random.default_rng(3)
    n = g.N * nphase
    x = rng.normal(size=n)
    y0 = rng.normal(size=n)
    yd = torch.as_tensor(y0.copy(), device="cuda")
    # both sides multiply the oracle's Jacobian, so only the product is compared
    A = o["val"]
    out = grid.spmv(torch.as_tensor(A.ravel(), device="cuda"), torch.as_tensor(x, device="cuda"), alpha, beta,
                    yd, transpose=transpose)
    ref, mag = oracle_spmv(o["row_ptr"], o["col_idx"], A, x, alpha, beta, y0, transpose=transpose)
    assert_scaled_close(out.cpu().numpy(), ref, mag, RTOL_SPMV, "spmv")


def test_spmv_beta_zero_ignores_y():
    O = ocp()
    g, s = W.tiny(3, 3, 3, seed=45)
    grid, o, (r, v, ff) = check_linearize(g, s)
    x = torch.ones(g.N * 3, dtype=torch.float64, device="cuda")
    y = torch.full((g.N * 3,), float("nan"), dtype=torch.float64, device="cuda")
    out = grid.spmv(torch.as_tensor(o["val"].ravel(), device="cuda"), x, 1.0, 0.0, y)
    assert torch.isfinite(out).all()


@pytest.mark.parametrize("nphase,shape", [(3, (4, 3, 3)), (2, (5, 4, 2)), (3, (1, 1, 1))])
def test_adjoint_vjp(nphase, shape):
    O = ocp()
    g, s = W.tiny(*shape, nphase=nphase, seed=46)
    rng = np.random.default_rng(4)
    lam = rng.normal(size=(g.N, nphase))
    o = orc(g, s, mode="all", lam=lam)
    grid = O.Grid(g)
    un, fn, uo, fo = dev_state(s)
    r, v, ff = grid.linearize(un, fn, uo, fo, s.dt, want_face_flux=True)
    out = grid.adjoint_vjp(un, fn, uo, fo, s.dt, v, ff, torch.as_tensor(lam.ravel(), device="cuda"))
    assert grid.status() == 0
    for k in ("unew", "uold", "lnk", "phi"):
        assert_scaled_close(out[k].cpu().numpy(), o["g_" + k], o["g_%s_mag" % k], RTOL_VJP, "g_" + k)


def test_adjoint_vjp_partial_outputs():
    O = ocp()
    g, s = W.tiny(3, 3, 2, seed=47)
    lam = np.random.default_rng(5).normal(size=(g.N, 3))
    o = orc(g, s, mode="all", lam=lam)
    grid = O.Grid(g)
    un, fn, uo, fo = dev_state(s)
    r, v, ff = grid.linearize(un, fn, uo, fo, s.dt, want_face_flux=True)
    out = grid.adjoint_vjp(un, fn, uo, fo, s.dt, v, ff, torch.as_tensor(lam.ravel(), device="cuda"),
                           want=("lnk",))
    assert set(out) == {"lnk"}
    assert_scaled_close(out["lnk"].cpu().numpy(), o["g_lnk"], o["g_lnk_mag"], RTOL_VJP, "g_lnk")


@pytest.mark.parametrize("nphase", [3, 2])
def test_well_rates(nphase):
    O = ocp()
    g, s = W.tiny(4, 4, 3, nphase=nphase, seed=48)
    o = orc(g, s)
    grid = O.Grid(g)
    un, fn, uo, fo = dev_state(s)
    q = grid.well_rates(un, fn).cpu().numpy().reshape(len(g.wells), nphase)
    for w, well in enumerate(g.wells):
        ref = o["well_q"][well.cells].sum(axis=0)
        np.testing.assert_allclose(q[w], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert np.abs(ref).max() > 0


# --------------------------------------------------------------- device status
def test_nonfinite_state_sets_status_and_clears():
    O = ocp()
    g, s = W.tiny(3, 2, 2, seed=49)
    grid = O.Grid(g)
    s.u_new[0, 5] = np.nan
    r, v, ff, st = gpu_linearize(grid, s)
    assert st == O.OCP_ERR_NONFINITE
    assert grid.status() == 0


def test_bad_flag_sets_status():
    O = ocp()
    g, s = W.tiny(3, 2, 2, seed=50)
    grid = O.Grid(g)
    s.flag_new[3] = 2
    r, v, ff, st = gpu_linearize(grid, s)
    assert st == O.OCP_ERR_INVALID_ARG


def test_invalid_arguments_are_rejected():
    O = ocp()
    g, s = W.tiny(2, 2, 2, seed=51)
    grid = O.Grid(g)
    un, fn, uo, fo = dev_state(s)
    with pytest.raises(O.OcpError) as e:
        grid.linearize(un, fn, uo, fo, 0.0)
    assert e.value.status == O.OCP_ERR_INVALID_ARG
    lib = O.load()
    assert lib.ocp_linearize(grid._h, None, None, None, None, 1.0, None, None, None, None) == O.OCP_ERR_INVALID_ARG
    x = torch.zeros(g.N * 3, dtype=torch.float64, device="cuda")
    with pytest.raises(O.OcpError):
        grid.spmv(torch.zeros(grid.nnzb * 9, dtype=torch.float64, device="cuda"), x, y=x)
    with pytest.raises(ValueError):
        grid.linearize(un[:-1], fn, uo, fo, 1.0)


# --------------------------------------------------------------- full sizes
def test_layered_box_full_size():
    """The 100x100x20 three-phase box (200 000 cells, 1 372 000 blocks), in
    the launch configuration the benchmark times, every entry compared."""
    g, s = W.layered_box()
    grid, o, (r, v, ff) = check_linearize(g, s)
    # and 50 products with it, on sampled rows
    rng = np.random.default_rng(6)
    x = rng.normal(size=g.N * 3)
    A = o["val"]
    y = grid.spmv(torch.as_tensor(A.ravel(), device="cuda"), torch.as_tensor(x, device="cuda")).cpu().numpy()
    rows = rng.choice(g.N, 2000, replace=False)
    ref, mag = oracle_spmv(o["row_ptr"], o["col_idx"], A, x, rows=rows)
    sel = (rows[:, None] * 3 + np.arange(3)).ravel()
    assert_scaled_close(y[sel], ref[sel], mag[sel], RTOL_SPMV, "spmv rows")


def test_channelised_oil_water_full_size_sampled():
    """The 60x220x85 oil-water model (1 122 000 cells, 2x2 blocks): every
    pattern index compared, plus 300 sampled rows (wells and corners
    included), each recomputed by the oracle on its window."""
    O = ocp()
    g, s = W.channelised_ow()
    grid = O.Grid(g)
    r, v, ff, st = gpu_linearize(grid, s, want_face_flux=False)
    assert st == 0
    rp, ci = grid.pattern()
    rp = rp.cpu().numpy()
    rng = np.random.default_rng(7)
    sample = list(rng.choice(g.N, 280, replace=False))
    sample += [0, g.N - 1] + [int(w.cells[0]) for w in g.wells] + [int(w.cells[-1]) for w in g.wells]
    for c in sample:
        h, st_, centre = window(g, s, c)
        o = orc(h, st_)
        assert_scaled_close(r[2 * c:2 * c + 2], o["R"][centre], o["R_mag"][centre], RTOL_R, "residual row %d" % c)
        blocks = v.reshape(-1, 2, 2)[rp[c]:rp[c + 1]]
        ob = o["val"][o["row_ptr"][centre]:o["row_ptr"][centre + 1]]
        om = o["val_mag"][o["row_ptr"][centre]:o["row_ptr"][centre + 1]]
        assert blocks.shape == ob.shape
        assert_scaled_close(blocks, ob, om, RTOL_J, "jacobian row %d" % c)
