"""A small backward-Euler Newton time stepper on top of the oracle (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

This is the FIM nonlinear iteration of Sec. 3.2.5 in its plainest form:
assemble the Jacobian and residual, solve the linear system (a library sparse
direct solve stands in for the paper's CPR-preconditioned Krylov solver),
update the primary variables, and test convergence.  It is only used on small
grids: for the Buckley-Leverett pin and for reference gradients.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .blackoil import segment, table_columns
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


def newton_step(spec, u_old, flag_old, dt, max_it=25, tol_p=1e-7, tol_s=1e-10, ds_max=0.2):
    """Solve R(u_new; u_old) = 0 for one step.  Returns (u_new, flag, out,
    iterations) where ``out`` is the oracle linearisation at the solution.
    An update that would change a saturation by more than ``ds_max`` is
    scaled down (the usual saturation chop of FIM simulators); with three
    phases the phase switch follows every update."""
    u = np.array(u_old, dtype=np.float64, copy=True)
    flag = np.array(flag_old, copy=True)
    nb = int(spec.nphase)
    for it in range(1, max_it + 1):
        o = linearize(spec, u, flag, u_old, flag_old, dt)
        A = bsr_to_scipy(o["row_ptr"], o["col_idx"], o["val"]).tocsc()
        du = spla.spsolve(A, -o["R"].ravel()).reshape(-1, nb).T
        big = np.max(np.abs(du[1])) if nb > 1 else 0.0
        if big > ds_max:
            du = du * (ds_max / big)
        u = u + du
        nsw = switch_phases(spec, u, flag)
        if nsw == 0 and np.max(np.abs(du[0])) < tol_p and np.max(np.abs(du[1])) < tol_s and \
                (nb < 3 or np.max(np.abs(du[2][flag == 0]), initial=0.0) < tol_s) and \
                (nb < 3 or np.max(np.abs(du[2][flag == 1]), initial=0.0) < tol_p):
            o = linearize(spec, u, flag, u_old, flag_old, dt)
            return u, flag, o, it
    raise RuntimeError("Newton did not converge in %d iterations" % max_it)
