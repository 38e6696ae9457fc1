"""One IMPEC step in pressure and component amounts (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

IMPEC (implicit pressure, explicit composition; among the solution methods
of the paper's introduction and Sec. 3.3) solves the pressure from the
volume balance at the new time level and then advances the component
amounts explicitly.  Written out for the black-oil model in the (P, N)
unknowns of Sec. 2.1:

  * at the old level (P^n, N^n): the phase split, and from it the phase
    mobilities, densities, capillary offsets p_a - P and R_s, frozen for the
    step, and the fluid volume V_f with its derivatives V_f,P and
    w_i = dV_f / dN_i;
  * fluxes linear in the new pressure: for every face and phase the upwind
    direction of the old potentials, F_a = T lambda_a,up (Phi_a,i - Phi_a,j)
    with Phi_a = P^{n+1} + (p_a - P)^n - gamma_a^n z; components as in the
    main path (dissolved gas with the oil's upwind R_s); well terms with the
    old mobilities at the new cell pressure, open where they were open;
  * the pressure equation of each cell, the volume balance at n+1 linearised
    about n and multiplied by V / dt:
      (V/dt)(phi^n - V_f^n) + (V/dt)(phi' - V_f,P) dP
        + sum_i w_i (sum_faces F_i(P^n + dP) - Q_i(P^n + dP)) = 0,
    affine in dP: a 7-point system A dP = -E_0 (one unknown per cell);
  * the explicit update N_i^{n+1} = N_i^n + (dt/V)(Q_i - sum_faces F_i) at
    P^{n+1}, conservative by construction.
A and E_0 come from dual numbers seeded on dP, so the matrix is the exact
derivative of the affine function above.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .blackoil import GRAV, RB_FT3, cell_properties
from .dual import D, where
from .linearize import bsr_pattern, depth, dims, face_pairs, transmissibility, well_index
from .pn import phase_split


def _old_level(spec, pn_old):
    """Phase split and cell properties at the old level (values only), and
    the fluid volume's derivatives by P and by each N_i."""
    nb = int(spec.nphase)
    L = nb + 1
    N = pn_old.shape[1]
    phi_ref = np.asarray(spec.phi, dtype=np.float64)
    u = [D.seed(pn_old[v], L, v) for v in range(L)]
    flag, sw, x, V_f, _ = phase_split(spec, u[0], u[1], u[2], u[3] if nb == 3 else None, phi_ref)
    c = lambda d: D.const(d.v, N, 1)
    pr = cell_properties(spec, c(u[0]), c(sw), c(x) if x is not None else None, flag, phi_ref)
    phi = cell_properties(spec, u[0], sw, x, flag, phi_ref)["phi"]
    return {"flag": flag, "pr": pr, "V_f": V_f.v, "V_f_P": V_f.g[:, 0], "w": V_f.g[:, 1:],
            "phi": phi.v, "phi_P": phi.g[:, 0]}


def _fluxes_and_sources(spec, pn_old, old, dP: D):
    """Component fluxes out of every cell summed over its faces, and the well
    sources, at P^{n+1} = P^n + dP (dP a dual number per cell)."""
    nb = int(spec.nphase)
    nx, ny, nz = dims(spec)
    N = nx * ny * nz
    k = dP.k
    pr = old["pr"]
    P1 = dP + pn_old[0]
    z = depth(spec)
    lnk = D.const(np.asarray(spec.lnk, dtype=np.float64), N, k)
    phases = ["w", "o", "g"][:nb]
    out = [D.const(0.0, N, k) for _ in range(nb)]
    out_v = np.zeros((N, nb))
    out_g = np.zeros((N, nb, k))
    out_m = np.zeros((N, nb))
    for d in range(3):
        fi, fj = face_pairs(spec, d)
        if len(fi) == 0:
            continue
        T = transmissibility(spec, d, lnk.take(fi), lnk.take(fj)).v
        dz_ij = z[fi] - z[fj]
        Pi, Pj = P1.take(fi), P1.take(fj)
        F = {}
        for a in phases:
            off_i = pr["p_" + a].v[fi] - pn_old[0][fi]
            off_j = pr["p_" + a].v[fj] - pn_old[0][fj]
            gamma = (pr["rho_" + a].v[fi] + pr["rho_" + a].v[fj]) * (0.5 * GRAV)
            # upwind by the old potentials
            dphi_old = (pr["p_" + a].v[fi] - pr["p_" + a].v[fj]) - gamma * dz_ij
            up_i = dphi_old >= 0.0
            lam_up = np.where(up_i, pr["lam_" + a].v[fi], pr["lam_" + a].v[fj])
            dphi = (Pi - Pj) + (off_i - off_j - gamma * dz_ij)
            F[a] = dphi * (T * lam_up)
            F["up_" + a] = up_i
        comp = [F["w"], F["o"]]
        if nb == 3:
            rs_up = np.where(F["up_o"], pr["Rs"].v[fi], pr["Rs"].v[fj])
            comp.append(F["g"] + F["o"] * rs_up)
        for e in range(nb):
            q = comp[e]
            np.add.at(out_v[:, e], fi, q.v)
            np.add.at(out_v[:, e], fj, -q.v)
            # the face's value depends on dP of its two cells: keep the whole
            # derivative row (columns are the cells' own dP slots)
            np.add.at(out_g[:, e, :], fi, q.g)
            np.add.at(out_g[:, e, :], fj, -q.g)
            np.add.at(out_m[:, e], fi, q.m)
            np.add.at(out_m[:, e], fj, q.m)
    flux = [D(out_v[:, e], out_g[:, e, :], out_m[:, e], np.abs(out_g[:, e, :])) for e in range(nb)]
    # wells at their fixed bottom-hole pressures, mobilities and open state frozen
    src_v = np.zeros((N, nb))
    src_g = np.zeros((N, nb, k))
    src_m = np.zeros((N, nb))
    for w in spec.wells:
        cw = np.asarray(w.cells, dtype=np.int64)
        if len(cw) == 0:
            continue
        WI = well_index(spec, w, lnk.take(cw)).v
        p_old = pn_old[0][cw]
        pc = P1.take(cw)
        if w.kind == 0:
            open_ = (p_old - w.p_bh) > 0.0
            qs = [(pc * -1.0 + w.p_bh) * np.where(open_, WI * pr["lam_" + a].v[cw], 0.0) for a in phases]
            if nb == 3:
                qs[2] = qs[2] + qs[1] * pr["Rs"].v[cw]
        else:
            open_ = (w.p_bh - p_old) > 0.0
            mob = pr["kr_w"].v[cw] * pr["imu_w"].v[cw] + pr["kr_o"].v[cw] * pr["imu_o"].v[cw]
            if nb == 3:
                mob = mob + pr["kr_g"].v[cw] * pr["imu_g"].v[cw]
            b_inj = (pr["b_w"] if w.phase == 0 else pr["b_g"]).v[cw]
            coef = np.where(open_, WI * mob * b_inj, 0.0)
            e_inj = 0 if w.phase == 0 else 2
            qs = [D.const(0.0, len(cw), k) if e != e_inj else (pc * -1.0 + w.p_bh) * coef for e in range(nb)]
        for e in range(nb):
            np.add.at(src_v[:, e], cw, qs[e].v)
            np.add.at(src_g[:, e, :], cw, qs[e].g)
            np.add.at(src_m[:, e], cw, qs[e].m)
    src = [D(src_v[:, e], src_g[:, e, :], src_m[:, e], np.abs(src_g[:, e, :])) for e in range(nb)]
    return flux, src


def pressure_system(spec, pn_old, dt):
    """The IMPEC pressure equation E(dP) = E_0 + A dP of every cell.
    Returns (A as scipy CSR on the 7-point pattern, E_0, magnitude scales of
    A's entries and of E_0, the old-level data)."""
    nb = int(spec.nphase)
    nx, ny, nz = dims(spec)
    N = nx * ny * nz
    pn_old = np.asarray(pn_old, dtype=np.float64).reshape(nb + 1, N)
    old = _old_level(spec, pn_old)
    # dP of every cell is its own variable: the flux of a face depends on the
    # two cells' dP, so seed each cell's dP in its own column (N columns)
    dP = D(np.zeros(N), np.eye(N), np.zeros(N), np.eye(N))
    flux, src = _fluxes_and_sources(spec, pn_old, old, dP)
    vdt = spec.dx * spec.dy * spec.dz / RB_FT3 / dt
    E = (old["phi"] - old["V_f"]) * vdt + dP * ((old["phi_P"] - old["V_f_P"]) * vdt)
    for e in range(nb):
        E = E + (flux[e] - src[e]) * old["w"][:, e]
    A = sp.csr_matrix(E.g)
    return A, E.v, np.abs(E.gm), E.m, old


def impec_step(spec, pn_old, dt):
    """One IMPEC step: the pressure system, its direct solve, and the explicit
    update.  Returns (pn_new, dP, A, E_0)."""
    nb = int(spec.nphase)
    nx, ny, nz = dims(spec)
    N = nx * ny * nz
    pn_old = np.asarray(pn_old, dtype=np.float64).reshape(nb + 1, N)
    A, E0, _, _, old = pressure_system(spec, pn_old, dt)
    dP = spla.spsolve(A.tocsc(), -E0)
    flux, src = _fluxes_and_sources(spec, pn_old, old, D.const(dP, N, 1))
    vdt = spec.dx * spec.dy * spec.dz / RB_FT3 / dt
    pn_new = pn_old.copy()
    pn_new[0] = pn_old[0] + dP
    for e in range(nb):
        pn_new[1 + e] = pn_old[1 + e] + (src[e].v - flux[e].v) / vdt
    return pn_new, dP, A, E0
