"""The black-oil equations in the paper's own unknowns, pressure and component
amounts, with the volume-balance equation (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Sec. 2.1 writes the model in the pressure P and the component amounts N_i
per bulk volume (eq. 4: N_i = phi sum_j S_j xi_j x_ij) and closes it with the
volume balance V_f = V_p: the fluid that the amounts occupy fills the pore
volume.  For black oil the phase split is explicit (no flash): with amounts in
surface volumes per bulk volume,
  * water occupies V_w = N_w / b_w(P);
  * if N_g <= R_s,sat(P) N_o all gas is dissolved: R_s = N_g / N_o, the oil is
    undersaturated and occupies V_o = N_o / b_o(P, R_s), no free gas;
  * otherwise R_s = R_s,sat(P), V_o = N_o / b_o(P) and the free gas
    N_g - R_s N_o occupies V_g = (N_g - R_s N_o) / b_g(P);
  * saturations are S_j = V_j / V_f with V_f = V_w + V_o + V_g.
The unknowns of a cell are (P, N_w, N_o[, N_g]) and its equations the
component balances (accumulation (N - N_old) V / dt, the same two-point
upwinded fluxes and well terms as ``oracle.linearize``, which depend on the
amounts only through the phase split) and the volume balance
r_v = phi(P) - V_f, which involves the cell alone.  Every derivative is
carried by dual numbers.

``eliminate_volume_row`` removes N_w with each cell's volume-balance row
(a Schur complement on the diagonal block): the remaining unknowns are
(P, N_o[, N_g]) with one block row per cell of the component equations.
"""
from __future__ import annotations

import numpy as np

from .blackoil import GRAV, RB_FT3, cell_properties, interp_on, segment, table_columns
from .dual import D, where
from .linearize import bsr_pattern, depth, dims, face_pairs, transmissibility, well_index


def phase_split(spec, P: D, Nw: D, No: D, Ng: D | None, phi_ref):
    """Black-oil phase split of Sec. 2.1.  Returns (flag, S_w, X, V_f, props0)
    with X = S_g (flag 0) or R_s (flag 1), and the PVT quantities used."""
    n, k = P.n, P.k
    three = spec.nphase == 3
    zero = D.const(0.0, n, k)
    if three:
        knots, cols = table_columns(spec)
        rs_sat = interp_on(knots, cols["Rs"], segment(knots, P.v), P)
        unsat = (No.v > 0.0) & (Ng.v <= rs_sat.v * No.v)
        flag = unsat.astype(np.int8)
        with np.errstate(all="ignore"):
            rs_un = Ng / No
        x_pvt = where(unsat, rs_un, zero)
    else:
        flag = np.zeros(n, dtype=np.int8)
        x_pvt = None
    # b_w, b_o, b_g and R_s do not depend on S_w: evaluate them first
    props0 = cell_properties(spec, P, zero, x_pvt, flag, phi_ref)
    V_w = Nw / props0["b_w"]
    V_o = No / props0["b_o"]
    V_f = V_w + V_o
    if three:
        with np.errstate(all="ignore"):
            V_g = where(flag == 1, zero, (Ng - props0["Rs"] * No) / props0["b_g"])
        V_f = V_f + V_g
        S_g = V_g / V_f
        X = where(flag == 1, props0["Rs"], S_g)
    else:
        X = None
    S_w = V_w / V_f
    return flag, S_w, X, V_f, props0


def natural_to_pn(spec, u, flag):
    """(P, N) of a natural state (p, S_w[, X]): N = phi S b (eq. 4) at p."""
    from .blackoil import masses
    nv = int(spec.nphase)
    N = u.shape[1]
    d = [D.const(u[v], N, 1) for v in range(nv)]
    pr = cell_properties(spec, d[0], d[1], d[2] if nv == 3 else None, flag, np.asarray(spec.phi, dtype=np.float64))
    m = masses(spec, pr)
    return np.stack([u[0]] + [mi.v for mi in m])


def linearize_pn(spec, pn_new, pn_old, dt):
    """Residual and Jacobian in the unknowns (P, N_w, N_o[, N_g]).

    Returns R (N, nb+1) with equations water, oil[, gas], volume balance;
    val (nnzb, nb+1, nb+1) with val[s, e, v] = dR[row, e] / du[col_idx[s], v];
    the magnitude scales, the pattern, and the phase-split flags."""
    nx, ny, nz = dims(spec)
    N = nx * ny * nz
    nb = int(spec.nphase)
    L = nb + 1
    pn_new = np.asarray(pn_new, dtype=np.float64).reshape(L, N)
    pn_old = np.asarray(pn_old, dtype=np.float64).reshape(L, N)
    phi_ref = np.asarray(spec.phi, dtype=np.float64)
    lnk = D.const(np.asarray(spec.lnk, dtype=np.float64), N, L)
    u = [D.seed(pn_new[v], L, v) for v in range(L)]
    flag, sw, x, V_f, _ = phase_split(spec, u[0], u[1], u[2], u[3] if nb == 3 else None, phi_ref)
    pr = cell_properties(spec, u[0], sw, x, flag, phi_ref)

    vol_rb = spec.dx * spec.dy * spec.dz / RB_FT3
    acc = [(u[1 + e] - pn_old[1 + e]) * (vol_rb / dt) for e in range(nb)]
    r_vol = pr["phi"] - V_f

    R = np.zeros((N, L))
    Rm = np.zeros((N, L))
    row_ptr, col_idx, slot = bsr_pattern(spec)
    val = np.zeros((len(col_idx), L, L))
    valm = np.zeros((len(col_idx), L, L))
    diag = row_ptr[:-1] + slot[3]
    cells = np.arange(N)

    def add_rows(rows, e, q: D, sign):
        np.add.at(R[:, e], rows, sign * q.v)
        np.add.at(Rm[:, e], rows, q.m)

    def add_block(blk, e, g, gm, sign):
        np.add.at(val[:, e, :], blk, sign * g)
        np.add.at(valm[:, e, :], blk, gm)

    for e in range(nb):
        add_rows(cells, e, acc[e], 1.0)
        add_block(diag, e, acc[e].g, acc[e].gm, 1.0)
    add_rows(cells, nb, r_vol, 1.0)
    add_block(diag, nb, r_vol.g, r_vol.gm, 1.0)

    # connection fluxes: two-point, phase-upwinded (as oracle.linearize)
    z = depth(spec)
    phases = ["w", "o", "g"][:nb]
    for d in range(3):
        fi, fj = face_pairs(spec, d)
        if len(fi) == 0:
            continue
        K2 = 2 * L
        Pi = {key: v.take(fi).embed(K2, 0) for key, v in pr.items() if v is not None}
        Pj = {key: v.take(fj).embed(K2, L) for key, v in pr.items() if v is not None}
        T = transmissibility(spec, d, lnk.take(fi).embed(K2, 0), lnk.take(fj).embed(K2, L))
        dz_ij = z[fi] - z[fj]
        F = {}
        for a in phases:
            gamma = (Pi["rho_" + a] + Pj["rho_" + a]) * (0.5 * GRAV)
            dphi = (Pi["p_" + a] - Pj["p_" + a]) - gamma * dz_ij
            up_i = dphi.v >= 0.0
            F[a] = T * where(up_i, Pi["lam_" + a], Pj["lam_" + a]) * dphi
            F["up_" + a] = up_i
        comp = [F["w"], F["o"]]
        if nb == 3:
            comp.append(F["g"] + where(F["up_o"], Pi["Rs"], Pj["Rs"]) * F["o"])
        blk_ii = diag[fi]
        blk_ij = row_ptr[fi] + slot[4 + d][fi]
        blk_ji = row_ptr[fj] + slot[2 - d][fj]
        blk_jj = diag[fj]
        for e in range(nb):
            q = comp[e]
            add_rows(fi, e, q, 1.0)
            add_rows(fj, e, q, -1.0)
            gi, gj = q.g[:, :L], q.g[:, L:]
            gmi, gmj = q.gm[:, :L], q.gm[:, L:]
            add_block(blk_ii, e, gi, gmi, 1.0)
            add_block(blk_ij, e, gj, gmj, 1.0)
            add_block(blk_ji, e, gi, gmi, -1.0)
            add_block(blk_jj, e, gj, gmj, -1.0)

    # wells at their fixed bottom-hole pressures (as oracle.linearize)
    for w in spec.wells:
        cw = np.asarray(w.cells, dtype=np.int64)
        if len(cw) == 0:
            continue
        P = {key: v.take(cw) for key, v in pr.items() if v is not None}
        WI = well_index(spec, w, lnk.take(cw))
        zero = D.const(0.0, len(cw), L)
        if w.kind == 0:
            open_ = (P["p_o"] - w.p_bh).v > 0.0
            qs = [where(open_, WI * P["lam_" + a] * (w.p_bh - P["p_o"]), zero) for a in phases]
            if nb == 3:
                qs[2] = qs[2] + P["Rs"] * qs[1]
        else:
            drive = w.p_bh - P["p_o"]
            open_ = drive.v > 0.0
            mob = P["kr_w"] * P["imu_w"] + P["kr_o"] * P["imu_o"]
            if nb == 3:
                mob = mob + P["kr_g"] * P["imu_g"]
            b_inj = P["b_w"] if w.phase == 0 else P["b_g"]
            q_inj = where(open_, WI * mob * b_inj * drive, zero)
            qs = [zero if e != (0 if w.phase == 0 else 2) else q_inj for e in range(nb)]
        for e in range(nb):
            add_rows(cw, e, qs[e], -1.0)
            add_block(diag[cw], e, qs[e].g, qs[e].gm, -1.0)

    return {"R": R, "R_mag": Rm, "val": val, "val_mag": valm, "row_ptr": row_ptr, "col_idx": col_idx,
            "flag": flag, "S_w": sw.v, "X": x.v if x is not None else None, "V_f": V_f.v}


def eliminate_volume_row(spec, o):
    """Schur complement of the volume-balance rows: each cell's row
    r_v + a . d = 0 gives d N_w = -(a_P dP + a_o dN_o [+ a_g dN_g] + r_v) / a_w,
    substituted into every block column of that cell.  Returns R3 (N, nb),
    val3 (nnzb, nb, nb) over (P, N_o[, N_g]), their magnitude scales, and the
    per-cell coefficients c = a / a_w and c_r = r_v / a_w."""
    nb = int(spec.nphase)
    R, val, row_ptr, col_idx = o["R"], o["val"], o["row_ptr"], o["col_idx"]
    N = R.shape[0]
    rows = np.repeat(np.arange(N), np.diff(row_ptr))
    diag = np.array([row_ptr[c] + np.flatnonzero(col_idx[row_ptr[c]:row_ptr[c + 1]] == c)[0] for c in range(N)])
    a = val[diag, nb, :]                       # d r_v / d (P, N_w, N_o[, N_g])
    c = a / a[:, 1:2]
    c_r = R[:, nb] / a[:, 1]
    keep = [0, 2, 3][:nb]
    cc = c[col_idx]                            # coefficients of each block's column cell
    val3 = val[:, :nb][:, :, keep] - val[:, :nb, 1:2] * cc[:, None, keep]
    mag3 = o["val_mag"][:, :nb][:, :, keep] + o["val_mag"][:, :nb, 1:2] * np.abs(cc[:, None, keep])
    corr = val[:, :nb, 1] * c_r[col_idx][:, None]
    R3 = R[:, :nb].copy()
    np.subtract.at(R3, rows, corr)
    R3m = o["R_mag"][:, :nb].copy()
    np.add.at(R3m, rows, np.abs(corr))
    return {"R": R3, "R_mag": R3m, "val": val3, "val_mag": mag3, "c": c, "c_r": c_r}


def newton_step_pn(spec, pn_old, dt, pn_start=None, max_it=30, tol_cnv=1e-9, tol_vol=1e-12):
    """One backward-Euler step in the (P, N) unknowns: Newton on the full
    system with a sparse direct solve (no chop: the phase split needs no
    variable switching).  Converged when every component residual divided by
    phi V / dt (V in reservoir barrels) is below tol_cnv and every volume
    residual below tol_vol.  Returns (pn, flag, linearisations)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    nb = int(spec.nphase)
    L = nb + 1
    pn = np.array(pn_old if pn_start is None else pn_start, dtype=np.float64, copy=True).reshape(L, -1)
    N = pn.shape[1]
    pv = np.asarray(spec.phi, dtype=np.float64) * (spec.dx * spec.dy * spec.dz / RB_FT3 / dt)
    for it in range(1, max_it + 1):
        o = linearize_pn(spec, pn, pn_old, dt)
        cnv = np.max(np.abs(o["R"][:, :nb]) / pv[:, None])
        if cnv < tol_cnv and np.max(np.abs(o["R"][:, nb])) < tol_vol:
            return pn, o["flag"], it
        A = sp.bsr_matrix((o["val"], o["col_idx"], o["row_ptr"]), shape=(N * L, N * L)).tocsc()
        d = spla.spsolve(A, o["R"].ravel()).reshape(N, L).T
        pn = pn - d
    raise RuntimeError("Newton did not converge in %d iterations" % max_it)
