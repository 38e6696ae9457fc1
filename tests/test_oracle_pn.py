"""Pins of the (P, N) oracle with the volume balance (Sec. 2.1, eq. 4):
the phase split inverts eq. 4, the residual equals the natural-variable
residual on consistent states, its Newton step is the natural Newton step
mapped through eq. 4, its Jacobian matches central differences, the volume-row
elimination reproduces the full solve, the saturated/undersaturated split
follows the dissolved-gas limit; and planted mistakes are caught."""
import importlib
import importlib.util
import os
import shutil
import sys

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2406_10862_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load(tmp_path=None, mutation=None, tag="base"):
    if mutation is None:
        import oracle.linearize as lin
        import oracle.pn as pn
        return lin, pn
    dst = tmp_path / ("oracle_pn_" + tag)
    shutil.copytree(os.path.join(ROOT, "oracle"), dst)
    f = dst / "pn.py"
    src = f.read_text()
    old, new = mutation
    assert src.count(old) == 1, old
    f.write_text(src.replace(old, new))
    name = "oracle_pn_mut_" + tag
    spec = importlib.util.spec_from_file_location(name, dst / "__init__.py", submodule_search_locations=[str(dst)])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    return importlib.import_module(name + ".linearize"), importlib.import_module(name + ".pn")


def _sib(pn, name):
    """A module of the same oracle package as ``pn`` (planted copies included)."""
    return importlib.import_module(pn.__name__.rsplit(".", 1)[0] + "." + name)


def _case(nphase):
    g, s = W.tiny(5, 4, 3, nphase=nphase, seed=3, frac_unsat=0.4 if nphase == 3 else 0.0, rs_hi=0.7)
    s.dt = 2.5          # a step other than one day, so that dt enters every term visibly
    return g, s


def _bsr(rp, ci, val):
    nb = val.shape[1]
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    return sp.bsr_matrix((val, ci, rp), shape=(n * nb, n * nb)).tocsc() if len(rows) else None


def pin_phase_split_inverts_eq4(lin, pn):
    D = pn.D
    for nphase in (2, 3):
        g, s = _case(nphase)
        N = g.N
        x = pn.natural_to_pn(g, s.u_new, s.flag_new)
        args = [D.const(x[v], N, 1) for v in range(nphase + 1)] + ([None] if nphase == 2 else [])
        flag, sw, X, vf, _ = pn.phase_split(g, *args, np.asarray(g.phi))
        assert np.array_equal(flag, s.flag_new)
        assert np.allclose(sw.v, s.u_new[1], rtol=0, atol=1e-14)
        if nphase == 3:
            assert np.allclose(X.v, s.u_new[2], rtol=1e-13, atol=1e-14)
        phi = g.phi * (1.0 + g.cr * (s.u_new[0] - g.p_ref))
        assert np.allclose(vf.v, phi, rtol=1e-14)


def pin_residual_equals_natural_on_consistent_states(lin, pn):
    for nphase in (2, 3):
        g, s = _case(nphase)
        o = pn.linearize_pn(g, pn.natural_to_pn(g, s.u_new, s.flag_new), pn.natural_to_pn(g, s.u_old, s.flag_old),
                            s.dt)
        ref = lin.linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt)
        assert np.all(np.abs(o["R"][:, :nphase] - ref["R"]) <= 1e-12 * ref["R_mag"])
        assert np.all(np.abs(o["R"][:, nphase]) <= 1e-14)


def pin_newton_step_is_the_natural_step(lin, pn):
    # on the volume-balance manifold the reduced (P, N) Newton step equals the
    # natural-variable Newton step mapped by eq. 4: dP = dp, dN = (dm/du) du
    for nphase in (2, 3):
        g, s = _case(nphase)
        o = pn.linearize_pn(g, pn.natural_to_pn(g, s.u_new, s.flag_new), pn.natural_to_pn(g, s.u_old, s.flag_old),
                            s.dt)
        red = pn.eliminate_volume_row(g, o)
        d_red = spla.spsolve(_bsr(o["row_ptr"], o["col_idx"], red["val"]), red["R"].ravel()).reshape(-1, nphase)
        ref = lin.linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt)
        d_nat = spla.spsolve(_bsr(ref["row_ptr"], ref["col_idx"], ref["val"]), ref["R"].ravel()).reshape(-1, nphase)
        assert np.allclose(d_red[:, 0], d_nat[:, 0], rtol=1e-9, atol=1e-9 * np.abs(d_nat[:, 0]).max())
        # dN_o (and dN_g): the natural step through dm/du of eq. 4 (dual numbers)
        bo = _sib(pn, "blackoil")
        cell_properties, masses, D = bo.cell_properties, bo.masses, pn.D
        nv = nphase
        u = [D.seed(s.u_new[v], nv, v) for v in range(nv)]
        m = masses(g, cell_properties(g, u[0], u[1], u[2] if nv == 3 else None, s.flag_new, np.asarray(g.phi)))
        for e in range(1, nv):
            dN = np.einsum("cv,cv->c", m[e].g, d_nat)
            assert np.allclose(d_red[:, e], dN, rtol=1e-8, atol=1e-9 * np.abs(dN).max())


def pin_central_differences(lin, pn):
    g, s = _case(3)
    x0 = pn.natural_to_pn(g, s.u_new, s.flag_new)
    xo = pn.natural_to_pn(g, s.u_old, s.flag_old)
    # move off the manifold a little so the volume row is not trivially zero
    x0[1] *= 1.001
    o = pn.linearize_pn(g, x0, xo, s.dt)
    rp, ci = o["row_ptr"], o["col_idx"]
    for c in (0, 7, 33, 59):
        for v in range(4):
            h = 1e-3 if v == 0 else 1e-7 * max(abs(x0[v, c]), 1e-3)
            xp, xm = x0.copy(), x0.copy()
            xp[v, c] += h
            xm[v, c] -= h
            fd = (pn.linearize_pn(g, xp, xo, s.dt)["R"] - pn.linearize_pn(g, xm, xo, s.dt)["R"]) / (2 * h)
            for r in range(g.N):
                blk = np.flatnonzero(ci[rp[r]:rp[r + 1]] == c)
                jac = o["val"][rp[r] + blk[0], :, v] if len(blk) else np.zeros(4)
                scale = np.abs(jac).max() + np.abs(fd[r]).max() + 1e-12
                noise = 1e-14 * o["R_mag"][r] / h        # rounding of the residual values, amplified by 1/h
                assert np.allclose(fd[r], jac, rtol=1e-5, atol=1e-6 * scale + noise), (c, v, r)


def pin_elimination_reproduces_the_full_solve(lin, pn):
    g, s = _case(3)
    x0 = pn.natural_to_pn(g, s.u_new, s.flag_new)
    x0[1] *= 1.002                      # off the manifold: the volume rows carry residuals
    o = pn.linearize_pn(g, x0, pn.natural_to_pn(g, s.u_old, s.flag_old), s.dt)
    d_full = spla.spsolve(_bsr(o["row_ptr"], o["col_idx"], o["val"]), o["R"].ravel()).reshape(-1, 4)
    red = pn.eliminate_volume_row(g, o)
    d_red = spla.spsolve(_bsr(o["row_ptr"], o["col_idx"], red["val"]), red["R"].ravel()).reshape(-1, 3)
    dNw = -(red["c"][:, 0] * d_red[:, 0] + red["c"][:, 2] * d_red[:, 1] + red["c"][:, 3] * d_red[:, 2]) \
        + red["c_r"]
    got = np.stack([d_red[:, 0], dNw, d_red[:, 1], d_red[:, 2]], axis=1)
    # two direct solves of a system with condition number ~1e8 agree to ~1e-8
    assert np.allclose(got, d_full, rtol=1e-6, atol=1e-7 * np.abs(d_full).max(axis=0))


def pin_dissolved_gas_limit_decides_the_split(lin, pn):
    bo = _sib(pn, "blackoil")
    interp, table_columns, D = bo.interp, bo.table_columns, pn.D
    g, s = _case(3)
    knots, cols = table_columns(g)
    P = np.full(4, 4800.0)
    rs_sat = interp(knots, cols["Rs"], D.const(P, 4, 1)).v
    No = np.full(4, 0.15)
    Ng = rs_sat * No * np.array([1.0 - 1e-9, 1.0 + 1e-9, 0.5, 2.0])
    Nw = np.full(4, 0.03)
    c = lambda a: D.const(a, 4, 1)
    flag, sw, X, vf, _ = pn.phase_split(g, c(P), c(Nw), c(No), c(Ng), np.full(4, 0.2))
    assert flag.tolist() == [1, 0, 1, 0]
    assert np.allclose(X.v[[0, 2]], (Ng / No)[[0, 2]], rtol=1e-15)      # R_s of the undersaturated oil
    assert X.v[1] >= 0.0 and X.v[1] < 1e-6 and X.v[3] > 0.01              # free gas: none at the limit


def pin_time_step_reaches_the_natural_solution(lin, pn):
    # both formulations solve the same discrete equations: one step from the
    # same state ends at the same pressures and amounts
    nt = _sib(pn, "newton")
    for nphase in (2, 3):
        g, s = W.tiny(6, 5, 3, nphase=nphase, seed=4, frac_unsat=0.3 if nphase == 3 else 0.0, rs_hi=0.7)
        x, flag, _ = pn.newton_step_pn(g, pn.natural_to_pn(g, s.u_old, s.flag_old), 1.0)
        u, f, _, _ = nt.newton_step(g, s.u_old, s.flag_old, 1.0)
        assert np.array_equal(flag, f)
        ref = pn.natural_to_pn(g, u, f)
        assert np.allclose(x[0], ref[0], rtol=0, atol=1e-6)
        for e in range(1, nphase + 1):
            assert np.allclose(x[e], ref[e], rtol=1e-9, atol=1e-12)


PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__[4:])
def test_pin(pin):
    lin, pn = _load()
    pin(lin, pn)


MUTATIONS = [
    ("r_vol = pr[\"phi\"] - V_f", "r_vol = pr[\"phi\"] + V_f"),                          # volume balance sign
    ("(Ng - props0[\"Rs\"] * No) / props0[\"b_g\"]", "Ng / props0[\"b_g\"]"),              # dissolved gas kept free
    ("unsat = (No.v > 0.0) & (Ng.v <= rs_sat.v * No.v)", "unsat = (No.v > 0.0) & (Ng.v >= rs_sat.v * No.v)"),
    ("acc = [(u[1 + e] - pn_old[1 + e]) * (vol_rb / dt)", "acc = [(u[1 + e] - pn_old[1 + e]) * (vol_rb * dt)"),
    ("S_w = V_w / V_f", "S_w = V_w / (V_f - V_w)"),
    ("c_r = R[:, nb] / a[:, 1]", "c_r = R[:, nb] / a[:, 0]"),
    ("V_o = No / props0[\"b_o\"]", "V_o = No * props0[\"b_o\"]"),
]


@pytest.mark.filterwarnings("ignore::scipy.sparse.linalg.MatrixRankWarning")
@pytest.mark.parametrize("k", range(len(MUTATIONS)))
def test_planted_mistake_is_caught(tmp_path, k):
    lin, pn = _load(tmp_path, MUTATIONS[k], "m%d" % k)
    failed = []
    for pin in PINS:
        try:
            with np.errstate(all="ignore"):
                pin(lin, pn)
        except (AssertionError, RuntimeError, ValueError, FloatingPointError, np.linalg.LinAlgError, IndexError,
                ZeroDivisionError):
            failed.append(pin.__name__)
    assert failed, "mutation %r passed every pin" % (MUTATIONS[k][0],)
