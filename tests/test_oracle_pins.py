"""Pins of the CPU oracle against facts fixed by the mathematics, not by itself.

Each test names the property it pins and the passage it follows.  Together
they are chosen so that a plausible slip anywhere in the oracle (a dropped
term, a wrong sign or index, a transposed block) fails at least one of them;
``test_oracle_mutations.py`` plants such slips and checks exactly that.
"""
import copy
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import blackoil as bo
from oracle.dual import D
from oracle.linearize import face_pairs, linearize
from oracle.spmv import bsr_spmv, bsr_to_dense, bsr_to_scipy
from paper_2406_10862_gb300 import workloads as W


def lin(g, s, **kw):
    return linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt, **kw)


def dense_J(o):
    return bsr_to_dense(o["row_ptr"], o["col_idx"], o["val"])


def flat_fluid(**over):
    """Incompressible, constant-property fluid and rock (flat tables)."""
    t = W.synthetic_tables()
    n = len(t["tab_p"])
    f = dict(tab_Bo=np.full(n, 1.25), tab_Bg=np.full(n, 0.001), tab_Rs=np.full(n, 900.0),
             tab_muo=np.full(n, 0.8), tab_mug=np.full(n, 0.02), cw=0.0, cr=0.0, co_under=0.0,
             pcow_max=0.0, pcgo_max=0.0)
    f.update(over)
    return f


# --------------------------------------------------------------------- P8
def test_table_interpolation_knots_and_linear_column():
    """Interpolation returns the knot values on knots, takes the right-hand
    piece there (its slope), and reproduces an exactly linear column (R_s =
    0.3 p) everywhere, including linear extrapolation beyond both ends."""
    g, _ = W.tiny(2, 1, 1)
    knots, cols = bo.table_columns(g)
    p = D.seed(knots.copy(), 1, 0)
    for name, y in cols.items():
        v = bo.interp(knots, y, p)
        np.testing.assert_allclose(v.v, y, rtol=2e-16, atol=0)
        k = bo.segment(knots, knots)
        slope = (y[k + 1] - y[k]) / (knots[k + 1] - knots[k])
        np.testing.assert_array_equal(v.g[:, 0], slope)
    ps = np.array([100.0, 400.0, 1234.5, 5000.0, 6400.0, 9000.0])
    rs = bo.interp(knots, cols["Rs"], D.seed(ps, 1, 0))
    np.testing.assert_allclose(rs.v, 0.3 * ps, rtol=1e-14)
    np.testing.assert_allclose(rs.g[:, 0], 0.3, rtol=1e-13)


def test_corey_values_and_stone_reductions():
    """Corey at the middle of the mobile range is k_max / 4 (exponent 2);
    Stone II reduces to the oil-water curve where S_g = 0 and to the
    oil-gas curve where S_w = S_wc (Aziz and Settari's normalisation)."""
    g3, _ = W.tiny(2, 1, 1)
    g2, _ = W.tiny(2, 1, 1, nphase=2)
    sw_mid = g3.swc + 0.5 * (1.0 - g3.swc - g3.sorw)
    sw = np.array([sw_mid, 0.2, 0.35, 0.6, g3.swc])
    n = len(sw)
    one = D.seed(sw, 1, 0)
    krw, kro, krg, _, _ = bo.relperm(g3, one, D.const(0.0, n, 1))
    assert krw.v[0] == pytest.approx(g3.krw_max / 4.0, rel=1e-15)
    krw2, kro2, _, _, _ = bo.relperm(g2, one, None)
    np.testing.assert_allclose(kro.v, kro2.v, rtol=1e-15, atol=1e-300)
    np.testing.assert_allclose(kro.g, kro2.g, rtol=1e-14, atol=1e-300)
    # S_w = S_wc: k_ro equals k_rog
    sg = np.array([0.0, 0.05, 0.2, 0.4, 0.7])
    sgd = D.seed(sg, 1, 0)
    _, kro3, krg3, _, _ = bo.relperm(g3, D.const(g3.swc, n, 1), sgd)
    s_og = np.clip((1.0 - sg - g3.swc - g3.sorg) / (1.0 - g3.swc - g3.sorg), 0, 1)
    np.testing.assert_allclose(kro3.v, g3.kro_cw * s_og ** 2, rtol=1e-14, atol=1e-300)
    # gas Corey in the middle of its range
    sgm = g3.sgc + 0.5 * (1.0 - g3.swc - g3.sgc - g3.sorg)
    _, _, krg4, _, _ = bo.relperm(g3, D.const(g3.swc, 1, 1), D.seed(np.array([sgm]), 1, 0))
    assert krg4.v[0] == pytest.approx(g3.krg_max / 4.0, rel=1e-15)


def test_clamps_have_zero_derivative_outside():
    g, _ = W.tiny(2, 1, 1)
    sw = D.seed(np.array([0.05, 0.95]), 1, 0)        # below S_wc, above 1 - S_orw
    krw, kro, _, _, _ = bo.relperm(g, sw, D.const(0.0, 2, 1))
    assert krw.v[0] == 0.0 and krw.g[0, 0] == 0.0
    assert kro.v[1] == 0.0 and kro.g[1, 0] == 0.0


def test_surface_densities():
    """At b = 1 and R_s = 0 each phase density is its surface density."""
    g, _ = W.tiny(1, 1, 1, **flat_fluid(tab_Bo=np.ones(20), tab_Rs=np.zeros(20),
                                        tab_Bg=np.full(20, 1.0 / W.synthetic_tables()["tab_p"][0])))
    g.bw_ref = 1.0
    p = D.seed(np.array([g.p_ref]), 3, 0)
    pr = bo.cell_properties(g, p, D.const(0.3, 1, 3), D.const(0.1, 1, 3), np.array([0]), np.array([0.2]))
    assert pr["rho_w"].v[0] == pytest.approx(g.rho_wsc, rel=1e-15)
    assert pr["rho_o"].v[0] == pytest.approx(g.rho_osc, rel=1e-15)


# --------------------------------------------------------------------- P1 / P2
@pytest.mark.parametrize("nphase,shape,seed", [(3, (4, 3, 2), 1), (2, (3, 3, 3), 2), (3, (5, 1, 3), 3)])
def test_global_mass_balance(nphase, shape, seed):
    """Closed boundaries: the fluxes cancel in pairs, so the sum of every
    component's residual over the grid is its accumulation minus its well
    sources (eq. 1 integrated over the whole domain)."""
    g, s = W.tiny(*shape, nphase=nphase, seed=seed)
    o = lin(g, s)
    lhs = o["R"].sum(axis=0)
    rhs = o["acc"].sum(axis=0) - o["well_q"].sum(axis=0)
    scale = o["R_mag"].sum(axis=0)
    assert np.all(np.abs(lhs - rhs) <= 1e-13 * scale)
    assert np.all(np.abs(o["face_flux"]).max() > 0)


def one_cell_copy(g, s, c):
    """The same cell alone (no neighbours), keeping its rock, state and the
    wells that perforate it."""
    h = copy.deepcopy(g)
    h.nx = h.ny = h.nz = 1
    h.lnk = g.lnk[[c]]
    h.phi = g.phi[[c]]
    h.top_depth = g.top_depth
    h.wells = []
    for w in g.wells:
        if c in set(int(x) for x in w.cells):
            ww = copy.deepcopy(w)
            ww.cells = np.array([0])
            h.wells.append(ww)
    st = W.State(u_new=s.u_new[:, [c]], flag_new=s.flag_new[[c]], u_old=s.u_old[:, [c]],
                 flag_old=s.flag_old[[c]], dt=s.dt)
    return h, st


@pytest.mark.parametrize("nphase", [3, 2])
def test_jacobian_column_sums(nphase):
    """Summed over all rows, a column block of J only keeps the cell's own
    accumulation and well derivatives (flux derivatives cancel between the
    two cells of every face).  The reference is the same cell linearised
    alone, where there are no faces at all."""
    g, s = W.tiny(3, 2, 2, nphase=nphase, seed=5)
    o = lin(g, s)
    J = dense_J(o)
    nb = nphase
    for c in range(g.N):
        colsum = J[:, c * nb:(c + 1) * nb].reshape(g.N, nb, nb).sum(axis=0)
        h, st = one_cell_copy(g, s, c)
        o1 = lin(h, st)
        np.testing.assert_allclose(colsum, o1["val"][0], rtol=1e-10, atol=1e-9 * np.abs(o1["val"][0]).max())


# --------------------------------------------------------------------- P3 / P4
@pytest.mark.parametrize("phase", ["w", "o", "g"])
def test_hydrostatic_equilibrium_has_no_potential_difference(phase):
    """With constant densities and a pressure column rising with depth by
    rho*g, the flow potential of that phase is the same in every cell, so
    its potential difference vanishes across every face (eq. 2: u = 0 when
    grad P = rho g grad z)."""
    g, s = W.tiny(2, 2, 6, seed=7, wells=False, **flat_fluid())
    z = g.top_depth + (np.arange(g.N) // (g.nx * g.ny) + 0.5) * g.dz
    probe = bo.cell_properties(g, D.seed(np.full(1, 4800.0), 3, 0), D.const(0.3, 1, 3),
                               D.const(0.1, 1, 3), np.array([0]), np.array([0.2]))
    rho = probe["rho_" + phase].v[0]
    p = 4000.0 + rho * bo.GRAV * z
    s.u_new[0] = p
    s.u_new[1] = 0.3
    s.u_new[2] = 0.1
    s.flag_new[:] = 0
    o = lin(g, s)
    for d in range(3):
        if (d, phase) in o["face_dphi"]:
            assert np.max(np.abs(o["face_dphi"][(d, phase)])) < 1e-9
    # the other phases are out of equilibrium vertically
    other = [a for a in "wog" if a != phase and abs(probe["rho_" + a].v[0] - rho) > 1.0]
    assert any(np.max(np.abs(o["face_dphi"][(2, a)])) > 1.0 for a in other)


def test_hydrostatic_water_column_residual_vanishes():
    """Only water mobile (S_w = 1 - S_orw, no free gas), water column in
    hydrostatic equilibrium, no wells, no time change: R = 0 in every cell."""
    g, s = W.tiny(3, 2, 5, seed=8, wells=False, **flat_fluid())
    z = g.top_depth + (np.arange(g.N) // (g.nx * g.ny) + 0.5) * g.dz
    s.u_new[0] = 3000.0 + g.rho_wsc * g.bw_ref * bo.GRAV * z
    s.u_new[1] = 1.0 - g.sorw
    s.u_new[2] = 0.0
    s.flag_new[:] = 0
    s.u_old, s.flag_old = s.u_new.copy(), s.flag_new.copy()
    o = lin(g, s)
    assert np.max(np.abs(o["R"]) / np.maximum(o["R_mag"], 1e-300)) < 1e-12


def test_uniform_state_is_steady():
    """Uniform state, one layer (no gravity head), no wells, no time change:
    every residual entry is exactly zero."""
    for nphase in (2, 3):
        g, s = W.tiny(4, 3, 1, nphase=nphase, seed=9, wells=False)
        s.u_new[:] = s.u_old[:, :1]
        s.flag_new[:] = s.flag_old[0]
        s.u_old, s.flag_old = s.u_new.copy(), s.flag_new.copy()
        o = lin(g, s)
        assert np.all(o["R"] == 0.0)


def test_compressible_hydrostatic_column_is_trapezoidal():
    """A compressible water column in continuous equilibrium, dp/dz = g rho(p)
    with rho = rho_sc b_ref (1 + c_w (p - p_ref)), has the closed form
    p(z) = p_ref - 1/c_w + (p_0 - p_ref + 1/c_w) exp(a (z - z_0)), a = g rho_sc
    b_ref c_w.  The face potential difference uses the mean of the two cell
    densities, i.e. the trapezoid rule for this ODE, so on this profile it is
    O(dz^3) -- tiny -- while a one-sided density would leave O(dz^2)."""
    g, s = W.tiny(1, 1, 8, seed=16, wells=False, **flat_fluid(cw=1e-4))
    z = g.top_depth + (np.arange(g.N) + 0.5) * g.dz
    a = bo.GRAV * g.rho_wsc * g.bw_ref * g.cw
    p0 = 3000.0
    s.u_new[0] = g.p_ref - 1.0 / g.cw + (p0 - g.p_ref + 1.0 / g.cw) * np.exp(a * (z - z[0]))
    s.u_new[1] = 1.0 - g.sorw
    s.u_new[2] = 0.0
    s.flag_new[:] = 0
    o = lin(g, s)
    dphi = np.abs(o["face_dphi"][(2, "w")])
    trap = a * a * bo.GRAV * g.rho_wsc * g.dz ** 3 / 12.0 * 2   # bound on the trapezoid error
    euler = 0.5 * a * bo.GRAV * g.rho_wsc * g.dz ** 2           # size of a one-sided error
    assert dphi.max() < trap + 1e-9
    assert euler > 1000 * (trap + 1e-9)


def test_capillary_spreading_direction():
    """Capillary pressure is P_cow = p_o - p_w (falling with S_w) and P_cgo =
    p_g - p_o (rising with S_g).  At uniform oil pressure and without gravity
    water and gas therefore each flow from the cell holding more of them to
    the cell holding less, and oil does not move."""
    g, s = W.tiny(2, 1, 1, seed=17, wells=False)
    s.u_new[0] = 4800.0
    s.u_new[1] = [0.45, 0.25]
    s.u_new[2] = [0.05, 0.25]
    s.flag_new[:] = 0
    o = lin(g, s)
    fw, fo, fg_tot = o["face_flux"][0, :, 0]
    assert fw > 0.0                      # water: cell 0 (wetter) -> cell 1
    assert fo == 0.0
    assert o["face_dphi"][(0, "g")][0] < 0.0   # gas potential higher in cell 1


# --------------------------------------------------------------------- P5
def test_single_phase_incompressible_pressure_block_is_laplacian():
    """Only oil mobile, constant properties, homogeneous k, one layer: the
    oil-equation / pressure block is lambda_o times the graph Laplacian whose
    weights are the closed-form transmissibilities C k A / h of a homogeneous
    medium; it is symmetric with zero row sums.  Because R_s is constant, the
    gas component moves with the oil: R_gas = R_s R_oil in every cell."""
    g, s = W.tiny(4, 3, 1, seed=10, wells=False, **flat_fluid())
    g.lnk[:] = math.log(50.0)
    s.u_new[1] = g.swc
    s.u_new[2] = 0.0
    s.flag_new[:] = 0
    s.u_old, s.flag_old = s.u_new.copy(), s.flag_new.copy()
    s.u_old[0] = s.u_new[0]
    o = lin(g, s)
    J = dense_J(o)
    nb = 3
    Jop = J[1::nb, 0::nb]
    lam_o = g.kro_cw * (1.0 / 1.25) * (1.0 / 0.8)
    Tx = 0.001127 * 50.0 * g.dy * g.dz / g.dx
    Ty = 0.001127 * 50.0 * g.dx * g.dz / g.dy
    Lap = np.zeros((g.N, g.N))
    for d, T in ((0, Tx), (1, Ty)):
        fi, fj = face_pairs(g, d)
        for a, b in zip(fi, fj):
            Lap[a, a] += T
            Lap[b, b] += T
            Lap[a, b] -= T
            Lap[b, a] -= T
    np.testing.assert_allclose(Jop, lam_o * Lap, rtol=1e-13, atol=1e-12 * lam_o * Tx)
    np.testing.assert_allclose(Jop, Jop.T, rtol=1e-13, atol=1e-12 * lam_o * Tx)
    np.testing.assert_allclose(o["R"][:, 2], 900.0 * o["R"][:, 1], rtol=1e-12,
                               atol=1e-12 * np.abs(o["R_mag"][:, 2]).max())


# --------------------------------------------------------------------- P6
def fd_jacobian(g, s, hp=1e-3, hs=1e-7, hrs=1e-3):
    N, nb = g.N, g.nphase
    Jfd = np.zeros((N * nb, N * nb))
    for c in range(N):
        for v in range(nb):
            h = hp if v == 0 else (hrs if (v == 2 and s.flag_new[c] == 1) else hs)
            sp, sm = copy.deepcopy(s), copy.deepcopy(s)
            sp.u_new[v, c] += h
            sm.u_new[v, c] -= h
            Jfd[:, c * nb + v] = (lin(g, sp)["R"].ravel() - lin(g, sm)["R"].ravel()) / (2 * h)
    return Jfd


@pytest.mark.parametrize("nphase,shape,seed", [(3, (3, 2, 2), 11), (2, (2, 2, 3), 12), (3, (1, 1, 4), 13)])
def test_dual_jacobian_matches_central_differences(nphase, shape, seed):
    """The dual-number Jacobian against central differences of the residual
    (h_p = 1e-3 psi, h_S = 1e-7), away from kinks; agreement to ~1e-7 of the
    row's size is what the O(h^2) truncation allows."""
    g, s = W.tiny(*shape, nphase=nphase, seed=seed)
    o = lin(g, s)
    for key, dphi in o["face_dphi"].items():
        assert np.min(np.abs(dphi)) > 1e-2, "state too close to an upwind switch"
    J = dense_J(o)
    Jfd = fd_jacobian(g, s)
    rowscale = np.abs(J).max(axis=1, keepdims=True)
    assert np.max(np.abs(J - Jfd) / rowscale) < 1e-6


H_CS = 1e-30     # complex step: no subtraction, so no truncation or cancellation error


@pytest.mark.parametrize("nphase,shape,seed", [(3, (3, 3, 2), 7), (2, (3, 2, 3), 8)])
def test_dual_jacobian_matches_complex_step(nphase, shape, seed):
    """The dual-number Jacobian against complex-step derivatives
    Im R(u + i h e_j) / h, exact to rounding for a residual that is analytic
    in u away from its branch points: every block entry within 1e-14 of its
    magnitude scale, and no derivative outside the 7-point block pattern
    (eqs. 1, 2 and 4; wells and mixed oil states included)."""
    g, s = W.tiny(*shape, nphase=nphase, seed=seed)
    N = g.N
    o = lin(g, s)
    rp, ci = o["row_ptr"], o["col_idx"]
    for c in range(N):
        for v in range(nphase):
            u = s.u_new.astype(complex).reshape(nphase, N).copy()
            u[v, c] += 1j * H_CS
            d = linearize(g, u.ravel(), s.flag_new, s.u_old, s.flag_old, s.dt)["R"].imag / H_CS
            for r in range(N):
                hit = np.nonzero(ci[rp[r]:rp[r + 1]] == c)[0]
                if len(hit) == 0:
                    assert not np.any(d[r]), (r, c, v)
                    continue
                k = rp[r] + hit[0]
                err = np.abs(d[r] - o["val"][k][:, v])
                assert np.all(err <= 1e-14 * o["val_mag"][k][:, v]), (r, c, v, err)


def test_vjp_parameter_gradients_match_complex_step():
    """lam^T dR/d(ln k, phi, u_old) of the dual-number VJP against complex
    steps of lam . R in each parameter of each cell (the derivatives the
    adjoint of a history match needs), within 1e-14 of their magnitude."""
    g, s = W.tiny(3, 2, 2, seed=15)
    N = g.N
    lam = np.random.default_rng(1).normal(size=(N, 3))
    o = lin(g, s, mode="all", lam=lam)
    for c in range(N):
        for name in ("lnk", "phi"):
            gg = copy.deepcopy(g)
            a = np.asarray(getattr(gg, name), dtype=complex).copy()
            a[c] += 1j * H_CS
            setattr(gg, name, a)
            cs = np.sum(lam * lin(gg, s)["R"].imag) / H_CS
            assert abs(cs - o["g_" + name][c]) <= 1e-14 * o["g_" + name + "_mag"][c], (name, c)
        for v in range(3):
            uo = s.u_old.astype(complex).reshape(3, N).copy()
            uo[v, c] += 1j * H_CS
            R = linearize(g, s.u_new, s.flag_new, uo.ravel(), s.flag_old, s.dt)["R"]
            cs = np.sum(lam * R.imag) / H_CS
            assert abs(cs - o["g_uold"][v, c]) <= 1e-14 * o["g_uold_mag"][v, c], ("u_old", v, c)


# --------------------------------------------------------------------- P9
def test_spmv_against_dense_and_library():
    g, s = W.tiny(4, 3, 2, seed=14)
    o = lin(g, s)
    rng = np.random.default_rng(0)
    x = rng.normal(size=g.N * 3)
    y0 = rng.normal(size=g.N * 3)
    y, m = bsr_spmv(o["row_ptr"], o["col_idx"], o["val"], x, alpha=-0.7, beta=0.3, y=y0)
    A = dense_J(o)
    np.testing.assert_allclose(y, -0.7 * (A @ x) + 0.3 * y0, rtol=0, atol=1e-15 * m.max())
    yt, mt = bsr_spmv(o["row_ptr"], o["col_idx"], o["val"], x, transpose=True)
    assert np.max(np.abs(yt - A.T @ x)) <= 1e-15 * mt.max()
    S = bsr_to_scipy(o["row_ptr"], o["col_idx"], o["val"])
    assert np.max(np.abs(S @ x - A @ x)) <= 1e-15 * m.max()


def test_bsr_pattern_counts():
    """nnzb = 7N - 2(ny nz + nx nz + nx ny) for the 7-point pattern, columns
    ascending in every row."""
    for shape in [(1, 1, 1), (2, 1, 1), (1, 1, 2), (3, 4, 5), (7, 1, 3)]:
        g, s = W.tiny(*shape, wells=False)
        o = lin(g, s)
        nx, ny, nz = shape
        assert o["row_ptr"][-1] == 7 * g.N - 2 * (ny * nz + nx * nz + nx * ny)
        for r in range(g.N):
            cols = o["col_idx"][o["row_ptr"][r]:o["row_ptr"][r + 1]]
            assert np.all(np.diff(cols) > 0) and r in cols


# --------------------------------------------------------------------- P10
def test_adjoint_dot_product_and_parameter_gradients():
    """<lam, J v> = <J^T lam, v>; and the vector-Jacobian products with
    respect to ln k, phi and the old state equal central differences of
    lam . R."""
    g, s = W.tiny(3, 2, 2, seed=15)
    rng = np.random.default_rng(1)
    lam = rng.normal(size=(g.N, 3))
    o = lin(g, s, mode="all", lam=lam)
    A = dense_J(o)
    v = rng.normal(size=g.N * 3)
    jtl = o["g_unew"].T.ravel()
    assert abs(lam.ravel() @ (A @ v) - jtl @ v) < 1e-13 * np.abs(lam.ravel()) @ (np.abs(A) @ np.abs(v))
    assert np.max(np.abs(jtl - A.T @ lam.ravel())) < 1e-12 * np.abs(A.T @ lam.ravel()).max()

    def f(gg, ss):
        return float(np.sum(lam * lin(gg, ss)["R"]))

    for name, h in (("lnk", 1e-6), ("phi", 1e-7)):
        for c in (0, 5, g.N - 1):
            gp, gm = copy.deepcopy(g), copy.deepcopy(g)
            getattr(gp, name)[c] += h
            getattr(gm, name)[c] -= h
            fd = (f(gp, s) - f(gm, s)) / (2 * h)
            assert fd == pytest.approx(o["g_" + name][c], rel=1e-6, abs=1e-9 * abs(fd) + 1e-6)
    for c in (1, 7):
        for vv, h in ((0, 1e-3), (1, 1e-7)):
            sp, sm = copy.deepcopy(s), copy.deepcopy(s)
            sp.u_old[vv, c] += h
            sm.u_old[vv, c] -= h
            fd = (f(g, sp) - f(g, sm)) / (2 * h)
            assert fd == pytest.approx(o["g_uold"][vv, c], rel=1e-6)


# ------------------------------------------------- undersaturated oil (R4)
def _oil_props(g, p, x, flag, sw=0.3):
    """Oil properties of cells at (p, S_w, X) as dual numbers in (p, X)."""
    n = len(p)
    P = D.seed(np.asarray(p, dtype=np.float64), 2, 0)
    X = D.seed(np.asarray(x, dtype=np.float64), 2, 1)
    pr = bo.cell_properties(g, P, D.const(sw, n, 2), X, np.full(n, flag, dtype=np.int8), np.full(n, 0.2))
    return pr, bo.masses(g, pr)


def test_undersaturated_oil_is_continuous_at_the_bubble_point():
    """At p = p_b(R_s) the undersaturated oil is the saturated oil without
    free gas: the same b_o, 1/mu_o, R_s, density, mobility and component
    amounts on either side of the phase switch (Sec. 2.1: the black-oil
    closure is explicit in the primary variables; reading R4), with nonzero
    oil compressibility and viscosibility so that a wrong bubble point, a
    wrong piece of the inverse table or a misplaced p - p_b shows."""
    g, _ = W.tiny(1, 1, 1, co_under=1e-5, cmu_under=2e-5)
    knots, cols = bo.table_columns(g)
    # knots (right-hand piece), interior points of pieces, both table ends
    p = np.concatenate([knots[:-1], 0.5 * (knots[:-1] + knots[1:]), [knots[-1], 417.25, 6123.5]])
    rs = 0.3 * p                                    # R_s,sat(p) of the exactly linear table
    un, mu = _oil_props(g, p, rs, 1)
    sa, ms = _oil_props(g, p, np.zeros_like(p), 0)
    for key in ("b_o", "imu_o", "Rs", "rho_o", "lam_o", "kr_o", "S_o"):
        np.testing.assert_allclose(un[key].v, sa[key].v, rtol=1e-13, atol=0, err_msg=key)
    for e in range(3):
        np.testing.assert_allclose(mu[e].v, ms[e].v, rtol=1e-13, atol=0, err_msg="m[%d]" % e)
    np.testing.assert_array_equal(un["S_g"].v, 0.0)
    np.testing.assert_array_equal(un["S_g"].g, 0.0)


@pytest.mark.parametrize("co,cmu", [(1e-5, 0.0), (1e-5, 2e-5), (3e-5, -1e-5)])
def test_undersaturated_oil_compressibility_closed_forms(co, cmu):
    """With the bubble point on a knot p_k (X = R_s at the knot, so p_b = p_k
    exactly) the undersaturated oil follows the closed forms of a constant
    compressibility c_o and viscosibility c_mu above it (reading R4):
      b_o = b_k (1 + c_o dp),  d ln b_o / dp = c_o / (1 + c_o dp),
      1/mu_o = (1/mu)_k (1 - c_mu dp), d ln(1/mu_o)/dp = -c_mu / (1 - c_mu dp),
    dp = p - p_k; and with respect to X, through dp_b/dX = 1/0.3 (the slope
    of the inverse of R_s = 0.3 p), the chain rule of the same forms on the
    table piece to the right of the knot."""
    g, _ = W.tiny(1, 1, 1, co_under=co, cmu_under=cmu)
    knots, cols = bo.table_columns(g)
    b, imu = cols["b_o"], cols["imu_o"]
    for k in (0, 7, 13):
        dp = np.array([0.0, 25.0, 400.0, 1750.0])
        p = knots[k] + dp
        x = np.full(len(p), cols["Rs"][k])
        pr, m = _oil_props(g, p, x, 1)
        sb = (b[k + 1] - b[k]) / (knots[k + 1] - knots[k])
        si = (imu[k + 1] - imu[k]) / (knots[k + 1] - knots[k])
        np.testing.assert_allclose(pr["b_o"].v, b[k] * (1.0 + co * dp), rtol=1e-14)
        np.testing.assert_allclose(pr["b_o"].g[:, 0] / pr["b_o"].v, co / (1.0 + co * dp), rtol=1e-12, atol=0)
        np.testing.assert_allclose(pr["imu_o"].v, imu[k] * (1.0 - cmu * dp), rtol=1e-14)
        np.testing.assert_allclose(pr["imu_o"].g[:, 0] / pr["imu_o"].v, -cmu / (1.0 - cmu * dp),
                                   rtol=1e-12, atol=1e-300)
        dpb = 1.0 / 0.3
        np.testing.assert_allclose(pr["b_o"].g[:, 1], dpb * (sb * (1.0 + co * dp) - co * b[k]), rtol=1e-12,
                                   atol=1e-18)
        np.testing.assert_allclose(pr["imu_o"].g[:, 1], dpb * (si * (1.0 - cmu * dp) + cmu * imu[k]),
                                   rtol=1e-12, atol=1e-18)
        # all gas dissolved: R_s is the unknown, no free gas, m_g = R_s m_o
        np.testing.assert_array_equal(pr["Rs"].v, x)
        np.testing.assert_array_equal(pr["Rs"].g, np.tile([0.0, 1.0], (len(p), 1)))
        np.testing.assert_allclose(m[2].v, x * m[1].v, rtol=1e-15)


# ------------------------------------------------------- Peaceman (R10)
def _radial_flow(nx, ny, dx, dy, k=100.0, h=20.0, p_e=3000.0, p_bh=2000.0):
    """Steady, incompressible, single-phase flow to one producer in the
    centre of a homogeneous 2-D grid whose outer ring of cells is held at
    p_e: the oracle's residual is affine in p here (flat tables, no rock or
    water compressibility, immobile water at S_wc, no gravity in one
    layer), so one Newton step from the uniform state with the ring's
    unknowns fixed is the exact discrete solution.  Returns the grid, the
    pressures, the oil production rate and q / (2 pi C k h lambda_o)."""
    m = 20
    g = W.make_grid(nx, ny, 1, np.full(nx * ny, math.log(k)), np.full(nx * ny, 0.2), [], nphase=2,
                    dx=dx, dy=dy, dz=h, tab_Bo=np.full(m, 1.25), tab_muo=np.full(m, 0.8), cw=0.0, cr=0.0,
                    pcow_max=0.0)
    cx, cy = nx // 2, ny // 2
    g.wells = [W.Well(kind=0, phase=0, p_bh=p_bh, cells=np.array([g.cell(cx, cy, 0)]))]
    N = g.N
    u = np.zeros((2, N))
    u[0] = p_e
    u[1] = g.swc
    flag = np.zeros(N, dtype=np.int8)
    o = linearize(g, u, flag, u, flag, 1.0)
    A = bsr_to_scipy(o["row_ptr"], o["col_idx"], o["val"]).tocsr()
    i, j = np.arange(N) % nx, np.arange(N) // nx
    ring = (i == 0) | (j == 0) | (i == nx - 1) | (j == ny - 1)
    free = np.repeat(~ring, 2)
    du = np.zeros(2 * N)
    du[free] = spla.spsolve(A[free][:, free].tocsc(), -o["R"].ravel()[free])
    u1 = u + du.reshape(N, 2).T
    o1 = linearize(g, u1, flag, u, flag, 1.0)
    assert np.max(np.abs(o1["R"][~ring])) < 1e-9 * np.max(np.abs(o1["R_mag"]))   # solved
    assert np.all(du[1::2] == 0.0)                                               # water stays put
    q = -o1["well_rate"][0, 1]
    lam_o = g.kro_cw / 1.25 / 0.8
    return g, u1[0], q, q / (2.0 * math.pi * bo.C_DARCY * k * h * lam_o), (cx, cy)


@pytest.mark.parametrize("nx,ny,dx,dy,tol", [(41, 41, 100.0, 100.0, 3e-3), (41, 61, 100.0, 60.0, 1e-2)])
def test_peaceman_well_reproduces_radial_flow(nx, ny, dx, dy, tol):
    """Peaceman's equivalent radius: with WI = 2 pi C k h / ln(r_o / r_w) and
    r_o = 0.14 sqrt(dx^2 + dy^2) (reading R10), the discrete pressure field
    around a producing well matches the continuous radial solution
    p(r) = p_bh + q / (2 pi C k h lambda) ln(r / r_w) away from the well
    block, because r_o is the radius at which the five-point scheme's
    well-block pressure sits on that solution (Peaceman's derivation; for
    square cells the lattice Green's function gives r_o = 0.1985 dx, and
    0.14 sqrt(2) dx = 0.1980 dx).  Differences between two far-field cells
    follow the same log law."""
    g, p, q, a, (cx, cy) = _radial_flow(nx, ny, dx, dy)
    assert q > 0.0
    rw = g.wells[0].rw
    for di, dj in [(3, 0), (4, 0), (6, 0), (3, 3), (4, 4), (5, 3), (-3, 0), (0, -4)]:
        r = math.hypot(di * dx, dj * dy)
        got = p[g.cell(cx + di, cy + dj, 0)] - 2000.0
        assert got == pytest.approx(a * math.log(r / rw), rel=tol), (di, dj)
    r1, r2 = 3 * dx, 6 * dx
    diff = p[g.cell(cx + 6, cy, 0)] - p[g.cell(cx + 3, cy, 0)]
    assert diff == pytest.approx(a * math.log(r2 / r1), rel=5 * tol)


# ----------------------------------------------------------- X10 at a tie
def test_upwind_flip_at_a_tie_changes_no_flux():
    """At a face whose potential difference is zero the flux vanishes
    whichever side is upwind (eq. 2: F = T lambda_up dphi), so flipping the
    upwind choice there (the oracle's ``up_flip``) leaves the residual and
    the face fluxes unchanged while the Jacobian's face blocks move to the
    other cell's mobility; on an untied face the flip changes the flux."""
    n = 20
    g, _ = W.tiny(3, 2, 6, seed=23, wells=False, **flat_fluid(cw=1e-4))
    z = g.top_depth + (np.arange(g.N) // (g.nx * g.ny) + 0.5) * g.dz
    # rho_w = rho_wsc b_w(p) is affine in p here, so the column at rest solves
    # p_k+1 - p_k = G (rho_k + rho_k+1) / 2 in closed form, G = g dz
    G, r0, c = bo.GRAV * g.dz, g.rho_wsc * g.bw_ref, g.cw
    a = 0.5 * G * r0 * c
    p = np.zeros(g.nz)
    p[0] = 3000.0
    for k in range(g.nz - 1):
        p[k + 1] = (p[k] * (1.0 + a) + G * r0 * (1.0 - c * g.p_ref)) / (1.0 - a)
    u = np.zeros((3, g.N))
    u[0] = p[np.arange(g.N) // (g.nx * g.ny)]
    u[1], u[2] = 0.5, 0.0
    f = np.zeros(g.N, dtype=np.int8)
    o = linearize(g, u, f, u, f, 1.0)
    dphi, mag = o["face_dphi"][(2, "w")], o["face_dphi_mag"][(2, "w")]
    assert np.all(np.abs(dphi) <= 64 * np.finfo(float).eps * mag)
    flip = {(2, "w"): np.ones(len(dphi), dtype=bool)}
    of = linearize(g, u, f, u, f, 1.0, up_flip=flip)
    np.testing.assert_allclose(of["R"], o["R"], rtol=0, atol=1e-12 * o["R_mag"].max())
    np.testing.assert_allclose(of["face_flux"], o["face_flux"], rtol=0, atol=1e-12 * o["face_flux_mag"].max())
    assert np.max(np.abs(of["val"] - o["val"]) / (o["val_mag"] + 1e-300)) > 1e-6
    # an untied face: the flip changes the flux
    g2, s2 = W.tiny(3, 2, 2, seed=4)
    o2 = lin(g2, s2)
    f2 = lin(g2, s2, up_flip={(0, "o"): np.ones(len(face_pairs(g2, 0)[0]), dtype=bool)})
    assert np.max(np.abs(f2["face_flux"][0, 1] - o2["face_flux"][0, 1])) > 1e-3 * np.max(np.abs(o2["face_flux"][0, 1]))
