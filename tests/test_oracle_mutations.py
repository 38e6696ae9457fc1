"""Planted mistakes in the oracle must be caught by its pins.

Each case copies the oracle package into a temporary directory, applies one
plausible slip to its source (a flipped sign, a dropped term, a transposed
block, a swapped upwind choice, ...), imports the copy under a fresh name and
runs a compact version of the pins on it.  The unmodified oracle passes every
pin; every mutant must fail at least one.  Mistakes are only ever planted in
this CPU copy.
"""
import copy
import importlib
import importlib.util
import math
import os
import shutil
import sys

import numpy as np
import pytest

from paper_2406_10862_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("linearize.py", 'dphi = (Pi["p_" + a] - Pj["p_" + a]) - gamma * dz_ij',
     'dphi = (Pi["p_" + a] - Pj["p_" + a]) + gamma * dz_ij'),                 # gravity sign
    ("linearize.py", "up_i = dphi.v >= 0.0", "up_i = dphi.v < 0.0"),           # downwind
    ("linearize.py", "add_rows(fj, e, q, -1.0)", "add_rows(fj, e, q, 1.0)"),   # flux sign
    ("linearize.py", "add_block(blk_ji, e, gi, gmi, -1.0)",
     "add_block(blk_ji, e, gj, gmj, -1.0)"),                                   # wrong operand
    ("linearize.py", "add_block(blk_ij, e, gj, gmj, 1.0)",
     "add_block(blk_ij, e, gi, gmi, 1.0)"),                                    # wrong operand
    ("linearize.py", 'comp.append(F["g"] + rs_up * F["o"])', 'comp.append(F["g"])'),  # dropped term
    ("linearize.py", 'gamma = (Pi["rho_" + a] + Pj["rho_" + a]) * (0.5 * GRAV)',
     'gamma = (Pi["rho_" + a] + Pi["rho_" + a]) * (0.5 * GRAV)'),              # wrong index
    ("linearize.py", "half_j = (0.5 * h) / kj", "half_j = (0.5 * h) * kj"),    # harmonic mean
    ("linearize.py", "(mn[e] - mo[e]) * (vol / RB_FT3) / dt", "(mn[e] - mo[e]) * (vol / RB_FT3) * dt"),
    ("linearize.py", '(pw - P["p_o"])', '(P["p_o"] - pw)'),                    # producer sign
    ("linearize.py", 'np.add.at(R[:, e], rows, sign * q.v)', 'np.add.at(R[:, e], rows, q.v)'),
    ("blackoil.py", "- (kr_w + kr_g))", ")"),                                   # Stone II term
    ("blackoil.py", 'out["p_w"] = p - pc_ow', 'out["p_w"] = p + pc_ow'),        # Pc sign
    ("blackoil.py", "return (x - knots[k]) * slope + y[k]", "return (x - knots[k + 1]) * slope + y[k]"),
    ("blackoil.py", 'm_o = pr["phi"] * pr["S_o"] * pr["b_o"]', 'm_o = pr["phi"] * pr["S_w"] * pr["b_o"]'),
    ("blackoil.py", 's_w = clamp01((sw - swc) / (1.0 - swc - sorw))',
     's_w = clamp01((sw - swc) / (1.0 - swc))'),                                # Corey end point
    ("dual.py", "g = self.g * o.v[:, None] + self.v[:, None] * o.g",
     "g = self.g * o.v[:, None]"),                                              # product rule term
    ("linearize.py", "return D(e, e[:, None] * a.g, ae, ae[:, None] * a.gm)",
     "return D(e, a.g, ae, ae[:, None] * a.gm)"),                              # d exp(x) = exp(x) dx
    ("dual.py", "dv = e * self.v ** (e - 1.0)", "dv = self.v ** (e - 1.0)"),   # power rule factor
    # the last entries name the pin that must catch them
    ("linearize.py", "r_o = 0.14 * np.sqrt(spec.dx ** 2 + spec.dy ** 2)",
     "r_o = 0.20 * np.sqrt(spec.dx ** 2 + spec.dy ** 2)", "pin_peaceman"),    # Peaceman radius
    ("blackoil.py", "(1.0 - spec.cmu_under * dp)", "(1.0 + spec.cmu_under * dp)",
     "pin_undersaturated"),                                                    # viscosibility sign
    ("blackoil.py", "(1.0 + spec.co_under * dp)", "(1.0 + 2.0 * spec.co_under * dp)",
     "pin_undersaturated"),                                                    # compressibility
    ("blackoil.py", "pb = interp_on(cols[\"Rs\"], knots, kr, x)",
     "pb = interp_on(cols[\"Rs\"], knots, kr, x) + 1.0", "pin_undersaturated"),   # bubble point off
]


def load_oracle(tmp_path, tag, mutation=None):
    dst = tmp_path / ("oracle_" + tag)
    shutil.copytree(os.path.join(ROOT, "oracle"), dst)
    if mutation is not None:
        fname, old, new = mutation[:3]
        f = dst / fname
        src = f.read_text()
        assert src.count(old) == 1, (fname, old)
        f.write_text(src.replace(old, new))
    name = "oracle_mut_" + tag
    spec = importlib.util.spec_from_file_location(name, dst / "__init__.py",
                                                  submodule_search_locations=[str(dst)])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    lin = importlib.import_module(name + ".linearize")
    newton = importlib.import_module(name + ".newton")
    bo = importlib.import_module(name + ".blackoil")
    return lin, newton, bo


def _flat(**over):
    n = 20
    f = dict(tab_Bo=np.full(n, 1.25), tab_Bg=np.full(n, 0.001), tab_Rs=np.full(n, 900.0),
             tab_muo=np.full(n, 0.8), tab_mug=np.full(n, 0.02), cw=0.0, cr=0.0, co_under=0.0,
             pcow_max=0.0, pcgo_max=0.0)
    f.update(over)
    return f


def run(lin, g, s, **kw):
    return lin.linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt, **kw)


def dense(o):
    nb = o["val"].shape[1]
    N = len(o["row_ptr"]) - 1
    A = np.zeros((N * nb, N * nb))
    for r in range(N):
        for k in range(o["row_ptr"][r], o["row_ptr"][r + 1]):
            c = o["col_idx"][k]
            A[r * nb:(r + 1) * nb, c * nb:(c + 1) * nb] = o["val"][k]
    return A


def pin_mass_balance(lin, newton, bo):
    g, s = W.tiny(3, 2, 2, seed=21)
    s.dt = 0.7
    o = run(lin, g, s)
    lhs = o["R"].sum(axis=0)
    rhs = o["acc"].sum(axis=0) - o["well_q"].sum(axis=0)
    return bool(np.all(np.abs(lhs - rhs) <= 1e-12 * o["R_mag"].sum(axis=0)))


def pin_fd(lin, newton, bo):
    g, s = W.tiny(2, 2, 2, seed=22)
    s.dt = 0.7
    o = run(lin, g, s)
    A = dense(o)
    N, nb = g.N, 3
    worst = 0.0
    for c in range(N):
        for v in range(nb):
            h = 1e-3 if v == 0 else (1e-3 if (v == 2 and s.flag_new[c] == 1) else 1e-7)
            sp, sm = copy.deepcopy(s), copy.deepcopy(s)
            sp.u_new[v, c] += h
            sm.u_new[v, c] -= h
            col = (run(lin, g, sp)["R"].ravel() - run(lin, g, sm)["R"].ravel()) / (2 * h)
            worst = max(worst, np.max(np.abs(col - A[:, c * nb + v]) / np.abs(A).max(axis=1)))
    return worst < 1e-6


def pin_hydrostatic(lin, newton, bo):
    g, s = W.tiny(2, 2, 5, seed=23, wells=False, **_flat())
    z = g.top_depth + (np.arange(g.N) // (g.nx * g.ny) + 0.5) * g.dz
    s.u_new[0] = 3000.0 + g.rho_wsc * g.bw_ref * bo.GRAV * z
    s.u_new[1] = 1.0 - g.sorw
    s.u_new[2] = 0.0
    s.flag_new[:] = 0
    s.u_old, s.flag_old = s.u_new.copy(), s.flag_new.copy()
    o = run(lin, g, s)
    return bool(np.max(np.abs(o["R"]) / np.maximum(o["R_mag"], 1e-300)) < 1e-12)


def pin_compressible_column(lin, newton, bo):
    g, s = W.tiny(1, 1, 6, seed=25, wells=False, **_flat(cw=1e-4))
    z = g.top_depth + (np.arange(g.N) + 0.5) * g.dz
    a = bo.GRAV * g.rho_wsc * g.bw_ref * g.cw
    s.u_new[0] = g.p_ref - 1.0 / g.cw + (3000.0 - g.p_ref + 1.0 / g.cw) * np.exp(a * (z - z[0]))
    s.u_new[1] = 1.0 - g.sorw
    s.u_new[2] = 0.0
    s.flag_new[:] = 0
    o = run(lin, g, s)
    return bool(np.max(np.abs(o["face_dphi"][(2, "w")])) < 1e-5)


def pin_capillary_direction(lin, newton, bo):
    g, s = W.tiny(2, 1, 1, seed=26, wells=False)
    s.u_new[0] = 4800.0
    s.u_new[1] = [0.45, 0.25]
    s.u_new[2] = [0.05, 0.25]
    s.flag_new[:] = 0
    o = run(lin, g, s)
    return bool(o["face_flux"][0, 0, 0] > 0.0 and o["face_dphi"][(0, "g")][0] < 0.0)


def pin_tables(lin, newton, bo):
    g, _ = W.tiny(1, 1, 1)
    knots, cols = bo.table_columns(g)
    ok = True
    for y in cols.values():
        ok = ok and np.allclose(bo.interp(knots, y, bo.D.seed(knots.copy(), 1, 0)).v, y, rtol=1e-15)
    ps = np.array([100.0, 1234.5, 9000.0])
    return bool(ok and np.allclose(bo.interp(knots, cols["Rs"], bo.D.seed(ps, 1, 0)).v, 0.3 * ps, rtol=1e-14))


def pin_laplacian(lin, newton, bo):
    g, s = W.tiny(3, 3, 1, seed=24, wells=False, **_flat())
    g.lnk[:] = math.log(50.0)
    s.u_new[1] = g.swc
    s.u_new[2] = 0.0
    s.flag_new[:] = 0
    s.u_old, s.flag_old = s.u_new.copy(), s.flag_new.copy()
    o = run(lin, g, s)
    A = dense(o)[1::3, 0::3]
    lam = g.kro_cw / 1.25 / 0.8
    Tx = 0.001127 * 50.0 * g.dy * g.dz / g.dx
    ok = abs(A[0, 1] + lam * Tx) < 1e-10 * lam * Tx and np.allclose(A, A.T, rtol=1e-12, atol=1e-9)
    ok = ok and np.allclose(o["R"][:, 2], 900.0 * o["R"][:, 1], rtol=1e-10, atol=1e-9)
    return bool(ok)


def pin_surface_density_and_stone(lin, newton, bo):
    g, _ = W.tiny(1, 1, 1)
    sw = bo.D.seed(np.array([0.3, 0.46]), 1, 0)
    kw, ko, kg, _, _ = bo.relperm(g, sw, bo.D.const(0.0, 2, 1))
    g2, _ = W.tiny(1, 1, 1, nphase=2)
    _, ko2, _, _, _ = bo.relperm(g2, sw, None)
    return bool(np.allclose(ko.v, ko2.v, rtol=1e-14) and abs(kw.v[1] - 0.1) < 1e-14)


def pin_buckley_leverett(lin, newton, bo):
    n = 60
    m = 20
    g = W.make_grid(n, 1, 1, np.full(n, math.log(100.0)), np.full(n, 0.2), [], nphase=2,
                    dx=1000.0 / n, dy=10.0, dz=10.0, tab_Bo=np.ones(m), tab_muo=np.full(m, 1.0),
                    cw=0.0, cr=0.0, bw_ref=1.0, muw=0.5, swc=0.0, sorw=0.0, krw_max=1.0,
                    kro_cw=1.0, pcow_max=0.0)
    g.wells = [W.Well(kind=1, phase=0, p_bh=1100.0, cells=np.array([0])),
               W.Well(kind=0, phase=0, p_bh=900.0, cells=np.array([n - 1]))]
    u = np.zeros((2, n))
    u[0] = 1000.0
    flag = np.zeros(n, dtype=np.int8)
    pv = 0.2 * 1000.0 * 100.0
    inj, dt = 0.0, 0.01
    try:
        for _ in range(200):
            u, flag, o, _ = newton.newton_step(g, u, flag, dt)
            q = o["well_q"][0, 0]
            if not q > 0:
                return False
            inj += q * dt * 5.614583
            if inj >= 0.3 * pv:
                break
            dt = min(0.3 * pv - inj + 1e-9, 0.3 * pv / 40) / (q * 5.614583)
    except Exception:
        return False
    r = 0.5
    sf = math.sqrt(r / (1 + r))
    S = np.linspace(1.0, sf, 4001)
    df = 2 * S * r * (1 - S) / (S * S + r * (1 - S) ** 2) ** 2
    qd = inj / pv
    xd = (np.arange(n) + 0.5) / n
    ex = np.interp(xd, qd * df, S, right=0.0)
    return bool(np.mean(np.abs(u[1] - ex)) < 0.04)


def pin_complex_step(lin, newton, bo):
    g, s = W.tiny(2, 2, 2, seed=22)
    o = run(lin, g, s)
    A = dense(o)
    M = np.abs(dense({"row_ptr": o["row_ptr"], "col_idx": o["col_idx"], "val": o["val_mag"]}))
    N, nb, h = g.N, 3, 1e-30
    for c in range(N):
        for v in range(nb):
            u = s.u_new.astype(complex).copy()
            u[v, c] += 1j * h
            col = lin.linearize(g, u, s.flag_new, s.u_old, s.flag_old, s.dt)["R"].ravel().imag / h
            if np.any(np.abs(col - A[:, c * nb + v]) > 1e-13 * M[:, c * nb + v]):
                return False
    # the adjoint's ln k gradient (transmissibility and well index)
    lam = np.random.default_rng(3).normal(size=(N, nb))
    o = run(lin, g, s, mode="all", lam=lam)
    for c in range(N):
        gg = copy.deepcopy(g)
        gg.lnk = np.asarray(gg.lnk, dtype=complex)
        gg.lnk[c] += 1j * h
        cs = np.sum(lam * run(lin, gg, s)["R"].imag) / h
        if abs(cs - o["g_lnk"][c]) > 1e-13 * o["g_lnk_mag"][c]:
            return False
    return True


def pin_undersaturated(lin, newton, bo):
    """Continuity at the bubble point and the closed forms above it, with
    c_mu != 0 (compact form of the pins in test_oracle_pins.py)."""
    g, _ = W.tiny(1, 1, 1, co_under=1e-5, cmu_under=2e-5)
    knots, cols = bo.table_columns(g)
    D = bo.D

    def props(p, x, flag):
        n = len(p)
        pr = bo.cell_properties(g, D.seed(p, 2, 0), D.const(0.3, n, 2), D.seed(x, 2, 1),
                                np.full(n, flag, dtype=np.int8), np.full(n, 0.2))
        return pr

    p = np.concatenate([knots[:-1], 0.5 * (knots[:-1] + knots[1:])])
    un, sa = props(p, 0.3 * p, 1), props(p, np.zeros_like(p), 0)
    ok = all(np.allclose(un[k].v, sa[k].v, rtol=1e-13, atol=0) for k in ("b_o", "imu_o", "rho_o", "lam_o"))
    k = 7
    dp = np.array([0.0, 400.0, 1750.0])
    pr = props(knots[k] + dp, np.full(3, cols["Rs"][k]), 1)
    ok = ok and np.allclose(pr["b_o"].v, cols["b_o"][k] * (1.0 + 1e-5 * dp), rtol=1e-14)
    ok = ok and np.allclose(pr["imu_o"].v, cols["imu_o"][k] * (1.0 - 2e-5 * dp), rtol=1e-14)
    return bool(ok)


def pin_peaceman(lin, newton, bo):
    """The pressure around a producer in a homogeneous 2-D grid with a
    fixed-pressure outer ring follows p_bh + q/(2 pi C k h lambda) ln(r/r_w)
    (compact form of the pin in test_oracle_pins.py)."""
    import scipy.sparse.linalg as spla
    from oracle.spmv import bsr_to_scipy
    n, m, dx = 31, 20, 100.0
    g = W.make_grid(n, n, 1, np.full(n * n, math.log(100.0)), np.full(n * n, 0.2), [], nphase=2,
                    dx=dx, dy=dx, dz=20.0, tab_Bo=np.full(m, 1.25), tab_muo=np.full(m, 0.8), cw=0.0, cr=0.0,
                    pcow_max=0.0)
    c = n // 2
    g.wells = [W.Well(kind=0, phase=0, p_bh=2000.0, cells=np.array([g.cell(c, c, 0)]))]
    N = g.N
    u = np.zeros((2, N))
    u[0], u[1] = 3000.0, g.swc
    flag = np.zeros(N, dtype=np.int8)
    o = lin.linearize(g, u, flag, u, flag, 1.0)
    A = bsr_to_scipy(o["row_ptr"], o["col_idx"], o["val"]).tocsr()
    i, j = np.arange(N) % n, np.arange(N) // n
    free = np.repeat(~((i == 0) | (j == 0) | (i == n - 1) | (j == n - 1)), 2)
    du = np.zeros(2 * N)
    du[free] = spla.spsolve(A[free][:, free].tocsc(), -o["R"].ravel()[free])
    u1 = u + du.reshape(N, 2).T
    q = -lin.linearize(g, u1, flag, u, flag, 1.0)["well_rate"][0, 1]
    a = q / (2.0 * math.pi * 0.001127 * 100.0 * 20.0 * (1.0 / 1.25 / 0.8))
    ok = True
    for di, dj in [(3, 0), (4, 0), (3, 3)]:
        r = math.hypot(di, dj) * dx
        ok = ok and abs((u1[0, g.cell(c + di, c + dj, 0)] - 2000.0) / (a * math.log(r / 0.25)) - 1.0) < 4e-3
    return bool(ok)


PINS = [pin_mass_balance, pin_fd, pin_complex_step, pin_hydrostatic, pin_compressible_column, pin_capillary_direction,
        pin_tables, pin_laplacian, pin_surface_density_and_stone,
        pin_buckley_leverett, pin_undersaturated, pin_peaceman]


def test_unmodified_oracle_passes_compact_pins(tmp_path):
    lin, newton, bo = load_oracle(tmp_path, "clean")
    for pin in PINS:
        assert pin(lin, newton, bo), pin.__name__


@pytest.mark.slow
@pytest.mark.parametrize("k", range(len(MUTATIONS)))
def test_planted_mistake_is_caught(tmp_path, k):
    lin, newton, bo = load_oracle(tmp_path, "m%d" % k, MUTATIONS[k])
    failed = []
    for pin in PINS:
        try:
            ok = pin(lin, newton, bo)
        except Exception:
            ok = False
        if not ok:
            failed.append(pin.__name__)
            break
    assert failed, "mutation %r passed every pin" % (MUTATIONS[k][1],)
    if len(MUTATIONS[k]) > 3:
        named = [p for p in PINS if p.__name__ == MUTATIONS[k][3]][0]
        try:
            ok = named(lin, newton, bo)
        except Exception:
            ok = False
        assert not ok, "mutation %r is not caught by %s" % (MUTATIONS[k][1], MUTATIONS[k][3])
