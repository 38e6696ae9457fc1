"""A small backward-Euler Newton time stepper on top of the oracle (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

This is the FIM nonlinear iteration of Sec. 3.2.5 in its plainest form:
assemble the Jacobian and residual, solve the linear system (a library sparse
direct solve stands in for the paper's CPR-preconditioned Krylov solver),
update the primary variables, and test convergence.  It is only used on small
grids: for the Buckley-Leverett pin, for reference gradients, and, with the
bottom-hole pressures as unknowns and rate-controlled wells, as the reference
of the library's well Newton loop.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .blackoil import RB_FT3, segment, table_columns
from .linearize import linearize
from .spmv import bsr_to_scipy


def switch_phases(spec, u, flag):
    """The saturated / undersaturated switch of the black-oil closure: a
    saturated cell whose S_g fell below zero holds no free gas and becomes
    undersaturated with R_s = R_s,sat(p); an undersaturated cell whose R_s
    exceeds R_s,sat(p) releases gas and becomes saturated with S_g = 0.
    Returns the number of switched cells (u and flag are updated in place)."""
    if spec.nphase != 3:
        return 0
    knots, cols = table_columns(spec)
    k = segment(knots, u[0])
    rs_sat = (u[0] - knots[k]) * ((cols["Rs"][k + 1] - cols["Rs"][k]) / (knots[k + 1] - knots[k])) + cols["Rs"][k]
    to_un = (flag == 0) & (u[2] < 0.0)
    to_sat = (flag == 1) & (u[2] > rs_sat)
    u[2, to_un] = rs_sat[to_un]
    u[2, to_sat] = 0.0
    flag[to_un] = 1
    flag[to_sat] = 0
    return int(to_un.sum() + to_sat.sum())


def chop(du, flag, ds_max):
    """Per-cell saturation chop: where a cell's saturation changes (S_w, and
    S_g in saturated cells) exceed ds_max, they are scaled down together to
    ds_max; pressure and R_s changes are kept."""
    du = du.copy()
    if du.shape[0] < 2:
        return du
    big = np.abs(du[1])
    if du.shape[0] == 3:
        big = np.maximum(big, np.where(flag == 0, np.abs(du[2]), 0.0))
    sc = np.where(big > ds_max, ds_max / np.where(big > 0.0, big, 1.0), 1.0)
    du[1] = du[1] * sc
    if du.shape[0] == 3:
        du[2] = np.where(flag == 0, du[2] * sc, du[2])
    return du


def newton_step(spec, u_old, flag_old, dt, max_it=25, tol_p=1e-7, tol_s=1e-10, ds_max=0.2):
    """Solve R(u_new; u_old) = 0 for one step.  Returns (u_new, flag, out,
    iterations) where ``out`` is the oracle linearisation at the solution.
    A cell whose saturations would change by more than ``ds_max`` has those
    changes scaled down (the usual saturation chop of FIM simulators); with
    three phases the phase switch follows every update."""
    u = np.array(u_old, dtype=np.float64, copy=True)
    flag = np.array(flag_old, copy=True)
    nb = int(spec.nphase)
    for it in range(1, max_it + 1):
        o = linearize(spec, u, flag, u_old, flag_old, dt)
        A = bsr_to_scipy(o["row_ptr"], o["col_idx"], o["val"]).tocsc()
        du = spla.spsolve(A, -o["R"].ravel()).reshape(-1, nb).T
        du = chop(du, flag, ds_max)
        u = u + du
        nsw = switch_phases(spec, u, flag)
        if nsw == 0 and np.max(np.abs(du[0])) < tol_p and np.max(np.abs(du[1])) < tol_s and \
                (nb < 3 or np.max(np.abs(du[2][flag == 0]), initial=0.0) < tol_s) and \
                (nb < 3 or np.max(np.abs(du[2][flag == 1]), initial=0.0) < tol_p):
            o = linearize(spec, u, flag, u_old, flag_old, dt)
            return u, flag, o, it
    raise RuntimeError("Newton did not converge in %d iterations" % max_it)


# ------------------------------------------------------------ wells as unknowns
def residual_norms(spec, o, dt, controls):
    """Convergence measures of a linearisation with well unknowns: for each
    equation e the largest |R_c,e| / (phi_c V_c / dt) (V in reservoir
    barrels: the residual as a change of surface volume per pore volume over
    the step), and the largest well residual, relative to max(|target|, 1)
    for rate-controlled wells and in psi for pressure-controlled ones."""
    vol_rb = spec.dx * spec.dy * spec.dz / RB_FT3
    pv = np.asarray(spec.phi, dtype=np.float64) * (vol_rb / dt)
    R = o["R"]
    out = [float(np.max(np.abs(R[:, e]) / pv)) for e in range(R.shape[1])]
    wr = 0.0
    for iw, (mode, _, target) in enumerate(controls):
        den = max(abs(target), 1.0) if mode == 1 else 1.0
        wr = max(wr, abs(o["well_res"][iw]) / den)
    return out, wr


def full_system(spec, o):
    """The Jacobian with the well rows and columns, [[A, B], [C, D]], as a
    scipy matrix; cell unknowns block-interleaved, then one p_bh per well."""
    nb = int(spec.nphase)
    N = int(spec.nx * spec.ny * spec.nz)
    nw = len(spec.wells)
    A = bsr_to_scipy(o["row_ptr"], o["col_idx"], o["val"])
    rows_b, cols_b, vals_b, rows_c, cols_c, vals_c = [], [], [], [], [], []
    k = 0
    for iw, w in enumerate(spec.wells):
        for c in np.asarray(w.cells, dtype=np.int64):
            for e in range(nb):
                rows_b.append(c * nb + e)
                cols_b.append(iw)
                vals_b.append(o["well_B"][k, e])
                rows_c.append(iw)
                cols_c.append(c * nb + e)
                vals_c.append(o["well_C"][k, e])
            k += 1
    B = sp.coo_matrix((vals_b, (rows_b, cols_b)), shape=(N * nb, nw))
    C = sp.coo_matrix((vals_c, (rows_c, cols_c)), shape=(nw, N * nb))
    Dm = sp.diags(o["well_D"])
    return sp.bmat([[A, B], [C, Dm]]).tocsc()


def newton_step_wells(spec, u_old, flag_old, dt, p_bh, controls, limits, max_it=30, tol_cnv=1e-9,
                      tol_well=1e-9, ds_max=0.2):
    """One backward-Euler step with the bottom-hole pressures as unknowns.

    Each iteration linearises at the current iterate, stops when the scaled
    residuals (``residual_norms``) are below the tolerances and the previous
    update switched nothing, else solves the full system, applies the
    saturation chop and the phase switch to the cells and the plain update to
    p_bh, and watches the well pressures: a rate-controlled producer whose
    p_bh fell below its limit, or injector whose p_bh rose above it, changes
    to pressure control at the limit for the rest of the step.
    Returns (u, flag, p_bh, controls, out, iterations)."""
    u = np.array(u_old, dtype=np.float64, copy=True)
    flag = np.array(flag_old, copy=True)
    p = np.array(p_bh, dtype=np.float64, copy=True)
    ctrl = [tuple(c) for c in controls]
    nb = int(spec.nphase)
    N = u.shape[1]
    nsw = 1
    for it in range(1, max_it + 1):
        o = linearize(spec, u, flag, u_old, flag_old, dt, p_bh=p, controls=ctrl)
        cnv, wr = residual_norms(spec, o, dt, ctrl)
        if nsw == 0 and max(cnv) < tol_cnv and wr < tol_well:
            return u, flag, p, ctrl, o, it
        rhs = np.concatenate([o["R"].ravel(), o["well_res"]])
        dx = spla.spsolve(full_system(spec, o), -rhs)
        du = chop(dx[:N * nb].reshape(-1, nb).T, flag, ds_max)
        u = u + du
        p = p + dx[N * nb:]
        nsw = switch_phases(spec, u, flag)
        for iw, w in enumerate(spec.wells):
            mode, ph, _ = ctrl[iw]
            if mode == 1 and ((w.kind == 0 and p[iw] < limits[iw]) or (w.kind == 1 and p[iw] > limits[iw])):
                ctrl[iw] = (0, ph, float(limits[iw]))
                p[iw] = limits[iw]
                nsw += 1
    raise RuntimeError("Newton did not converge in %d iterations" % max_it)
