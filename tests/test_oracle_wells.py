"""Pins of the oracle's well unknowns (bottom-hole pressures as unknowns, rate
and pressure controls, the "w" rows and columns of the Jacobian, Sec. 3.4.1)
and of its Newton loop with well controls: identity with the fixed-pressure
wells, central differences of the residual program, global mass balance,
rate targets met, the pressure-limit switch, and planted mistakes."""
import importlib.util
import os
import shutil

import numpy as np
import pytest

from paper_2406_10862_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load(tmp_path=None, mutation=None, tag="base"):
    """The oracle package, or a copy with one planted mistake in linearize.py."""
    if mutation is None:
        import oracle.linearize as lin
        import oracle.newton as nt
        return lin, nt
    dst = tmp_path / ("oracle_w_" + tag)
    shutil.copytree(os.path.join(ROOT, "oracle"), dst)
    f = dst / "linearize.py"
    src = f.read_text()
    old, new = mutation
    assert src.count(old) == 1, old
    f.write_text(src.replace(old, new))
    name = "oracle_w_mut_" + tag
    spec = importlib.util.spec_from_file_location(name, dst / "__init__.py", submodule_search_locations=[str(dst)])
    mod = importlib.util.module_from_spec(spec)
    import sys
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    lin = importlib.import_module(name + ".linearize")
    nt = importlib.import_module(name + ".newton")
    return lin, nt


def _case(nphase=3):
    g, s = W.tiny(6, 5, 3, nphase=nphase, seed=4, frac_unsat=0.3 if nphase == 3 else 0.0)
    return g, s


CTRL3 = [(1, 1, 200.0), (1, 2, 500.0)]       # producer: 200 of oil; injector: 500 of gas (surface units)
LIM3 = [1000.0, 8000.0]


def pin_bhp_mode_is_the_fixed_pressure_well(lin, nt):
    for nphase in (2, 3):
        g, s = _case(nphase)
        ref = lin.linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, 1.0)
        p = np.array([w.p_bh for w in g.wells])
        o = lin.linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, 1.0, p_bh=p)
        assert np.array_equal(o["R"], ref["R"]) and np.array_equal(o["val"], ref["val"])
        assert np.all(o["well_res"] == 0.0) and np.all(o["well_D"] == 1.0) and np.all(o["well_C"] == 0.0)


def pin_central_differences(lin, nt):
    # dR_cell/dp_bh, dR_w/dp_bh and dR_w/du_cell of the program, by central
    # differences of its values
    g, s = _case()
    p = np.array([4300.0, 5300.0])
    ctrl = [(1, 1, 150.0), (1, 2, 400.0)]
    o = lin.linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, 1.0, p_bh=p, controls=ctrl)
    h = 1e-3
    k0 = 0
    for iw, w in enumerate(g.wells):
        pp, pm = p.copy(), p.copy()
        pp[iw] += h
        pm[iw] -= h
        op = lin.linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, 1.0, p_bh=pp, controls=ctrl)
        om = lin.linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, 1.0, p_bh=pm, controls=ctrl)
        dR = (op["R"] - om["R"]) / (2 * h)
        dW = (op["well_res"][iw] - om["well_res"][iw]) / (2 * h)
        cells = np.asarray(w.cells)
        B = o["well_B"][k0:k0 + len(cells)]
        assert np.allclose(dR[cells], B, rtol=1e-6, atol=1e-9 * np.abs(B).max())
        others = np.setdiff1d(np.arange(g.N), cells)
        assert np.all(dR[others] == 0.0)
        assert dW == pytest.approx(o["well_D"][iw], rel=1e-6)
        # dR_w/du at each perforated cell, every variable
        for j, c in enumerate(cells):
            for v in range(3):
                up, um = s.u_new.copy(), s.u_new.copy()
                dv = 1e-3 if v == 0 else 1e-7
                up[v, c] += dv
                um[v, c] -= dv
                wp = lin.linearize(g, up, s.flag_new, s.u_old, s.flag_old, 1.0, p_bh=p, controls=ctrl)["well_res"][iw]
                wm = lin.linearize(g, um, s.flag_new, s.u_old, s.flag_old, 1.0, p_bh=p, controls=ctrl)["well_res"][iw]
                fd = (wp - wm) / (2 * dv)
                ref = o["well_C"][k0 + j, v]
                assert fd == pytest.approx(ref, rel=1e-5, abs=1e-6 * (abs(ref) + 1e-3))
        k0 += len(cells)


def _solve(nt, g, s, ctrl, lim, p0):
    return nt.newton_step_wells(g, s.u_old, s.flag_old, 1.0, np.array(p0), ctrl, lim)


def pin_rate_targets_and_mass_balance(lin, nt):
    g, s = _case()
    u, f, p, ctrl, o, it = _solve(nt, g, s, CTRL3, LIM3, [3000.0, 6000.0])
    assert ctrl == CTRL3                                   # no limit reached
    assert -o["well_rate"][0, 1] == pytest.approx(200.0, rel=1e-9)
    assert o["well_rate"][1, 2] == pytest.approx(500.0, rel=1e-9)
    # closed boundaries, conservative fluxes: summed over the cells, the
    # residual is what accumulates minus what the wells put in
    acc = o["acc"].sum(axis=0)
    src = o["well_rate"].sum(axis=0)
    scale = np.abs(o["acc"]).sum(axis=0) + np.abs(o["well_rate"]).sum(axis=0) + np.abs(o["R"]).sum(axis=0)
    assert np.all(np.abs(o["R"].sum(axis=0) - (acc - src)) <= 1e-12 * scale)
    # and at the solution that imbalance is within the convergence tolerance
    pv = g.phi * (g.dx * g.dy * g.dz / 5.614583)
    assert np.all(np.abs(acc - src) <= 1e-9 * pv.sum())


def pin_pressure_limit_switch(lin, nt):
    # an oil target the producer cannot reach above 4000 psi
    g, s = _case()
    ctrl = [(1, 1, 1e6), (0, 2, 5100.0)]
    u, f, p, c, o, it = _solve(nt, g, s, ctrl, [4000.0, 8000.0], [4500.0, 5100.0])
    assert c[0] == (0, 1, 4000.0) and p[0] == 4000.0
    assert 0.0 < -o["well_rate"][0, 1] < 1e6
    assert p[1] == pytest.approx(5100.0, abs=1e-9)


def pin_pressure_controls_match_the_fixed_pressure_newton(lin, nt):
    g, s = _case()
    p0 = [w.p_bh for w in g.wells]
    ctrl = [(0, 1, w.p_bh) for w in g.wells]
    u, f, p, c, o, it = _solve(nt, g, s, ctrl, [0.0, 1e9], p0)
    u2, f2, o2, it2 = nt.newton_step(g, s.u_old, s.flag_old, 1.0)
    assert np.array_equal(f, f2)
    assert np.allclose(u, u2, rtol=1e-9, atol=1e-9)


PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__[4:])
def test_pin(pin):
    lin, nt = _load()
    pin(lin, nt)


MUTATIONS = [
    ('sgn = -1.0 if w.kind == 0 else 1.0', 'sgn = 1.0'),                         # production sign
    ('w_B.append(np.stack([-qs[e].g[:, L]', 'w_B.append(np.stack([qs[e].g[:, L]'),  # B sign
    ('w_D[iw] = sgn * q.g[:, L].sum()', 'w_D[iw] = q.g[:, L].sum()'),              # D sign
    ('c_blk[:, :nv] = sgn * q.g[:, :nv]', 'c_blk[:, :nv] = q.g[:, :nv]'),          # C sign
    ('w_res[iw] = sgn * q.v.sum() - target', 'w_res[iw] = sgn * q.v.sum() + target'),
    ('pw = D.seed(np.full(n_w, p_bh[iw]), Lw, L)', 'pw = D.const(np.full(n_w, p_bh[iw]), n_w, Lw)'),
]


@pytest.mark.filterwarnings("ignore::scipy.sparse.linalg.MatrixRankWarning")
@pytest.mark.parametrize("k", range(len(MUTATIONS)))
def test_planted_mistake_is_caught(tmp_path, k):
    lin, nt = _load(tmp_path, MUTATIONS[k], "m%d" % k)
    failed = []
    for pin in PINS:
        try:
            pin(lin, nt)
        except (AssertionError, RuntimeError, ValueError, FloatingPointError, np.linalg.LinAlgError):
            failed.append(pin.__name__)
    assert failed, "mutation %r passed every pin" % (MUTATIONS[k][0],)
