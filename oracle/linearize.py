"""One FIM Newton linearisation of the black-oil equations, written out plainly.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

What is computed is the discrete residual of the component mass balance
(eq. 1 with the diffusion term dropped, Darcy velocities by eq. 2, component
amounts by eq. 4, saturations closing to one) after a backward-Euler step and
a two-point flux approximation on a Cartesian grid, and its exact Jacobian
with respect to the unknowns at the new time level.  The Jacobian is *not*
derived by hand here: every contribution is evaluated in forward-mode dual
numbers (``oracle.dual``), so it is the derivative of exactly the residual
program below.  The four stages follow the paper's split of the reservoir
into cell terms (Bulk / ACCU, Sec. 3.2.3), connection terms (BulkConn,
Sec. 3.2.4) and well terms (AllWells, Sec. 3.2.4); their assembly into
block rows follows the block-CSR matrix of the LinearSystem module
(Sec. 3.3.3).

Layouts (shared with the library's C interface):
* state ``u``: shape (nv, N), variable-major (p, S_w[, X]); ``flag`` (N,) int8;
* residual: shape (N, nb), equations water, oil[, gas] -- flattened it is the
  block-interleaved vector ``r[nb*c + e]``;
* Jacobian: block-CSR, ``row_ptr`` (N+1), ``col_idx`` (nnzb), ``val``
  (nnzb, nb, nb) with ``val[s, e, v] = dR[row, e] / du[col_idx[s], v]``;
  within a row the columns ascend (c-nx*ny, c-nx, c-1, c, c+1, c+nx, c+nx*ny).
"""
from __future__ import annotations

import numpy as np

from .blackoil import C_DARCY, GRAV, RB_FT3, cell_properties, masses
from .dual import D, where


# ------------------------------------------------------------------- geometry
def dims(spec):
    return int(spec.nx), int(spec.ny), int(spec.nz)


def cell_ijk(spec):
    nx, ny, nz = dims(spec)
    c = np.arange(nx * ny * nz)
    return c % nx, (c // nx) % ny, c // (nx * ny)


def depth(spec):
    """Cell-centre depth, positive downward."""
    _, _, kk = cell_ijk(spec)
    return spec.top_depth + (kk + 0.5) * spec.dz


def face_pairs(spec, d):
    """(i, j) cell pairs of the faces normal to direction d (0=x, 1=y, 2=z),
    j being the + neighbour of i."""
    nx, ny, nz = dims(spec)
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    if d == 0:
        return idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel()
    if d == 1:
        return idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel()
    return idx[:-1, :, :].ravel(), idx[1:, :, :].ravel()


def transmissibility(spec, d, lnk_i: D, lnk_j: D) -> D:
    """Two-point transmissibility: the series (harmonic) combination of the
    two half-cell conductances, C * A / (h/(2 k_i) + h/(2 k_j))."""
    dx, dy, dz = spec.dx, spec.dy, spec.dz
    h, area = [(dx, dy * dz), (dy, dx * dz), (dz, dx * dy)][d]
    ki = _exp(lnk_i)
    kj = _exp(lnk_j)
    if d == 2:
        ki = ki * spec.kz_over_kx
        kj = kj * spec.kz_over_kx
    half_i = (0.5 * h) / ki
    half_j = (0.5 * h) / kj
    return (C_DARCY * area) / (half_i + half_j)


def _exp(a: D) -> D:
    e = np.exp(a.v)
    ae = np.abs(e)                       # the magnitude (e itself for real a)
    return D(e, e[:, None] * a.g, ae, ae[:, None] * a.gm)


def well_index(spec, well, lnk_c: D) -> D:
    """Peaceman's well index for a vertical well through an isotropic cell,
    with equivalent radius r_o = 0.14 sqrt(dx^2 + dy^2):
    WI = C * 2 pi k h / (ln(r_o / r_w) + skin)."""
    r_o = 0.14 * np.sqrt(spec.dx ** 2 + spec.dy ** 2)
    geom = C_DARCY * 2.0 * np.pi * spec.dz / (np.log(r_o / well.rw) + well.skin)
    return _exp(lnk_c) * geom


# ------------------------------------------------------------------ BSR layout
def bsr_pattern(spec):
    """row_ptr, col_idx of the 7-point pattern and the slot of each neighbour
    inside its row (slot arrays hold -1 where the neighbour does not exist)."""
    nx, ny, nz = dims(spec)
    N = nx * ny * nz
    i, j, k = cell_ijk(spec)
    has = [k > 0, j > 0, i > 0, np.ones(N, bool), i < nx - 1, j < ny - 1, k < nz - 1]
    offs = [-nx * ny, -nx, -1, 0, 1, nx, nx * ny]
    cnt = np.sum(np.stack(has), axis=0)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(cnt)
    col_idx = np.zeros(row_ptr[-1], dtype=np.int64)
    slot = np.full((7, N), -1, dtype=np.int64)
    pos = np.zeros(N, dtype=np.int64)
    c = np.arange(N)
    for s in range(7):
        h = has[s]
        slot[s, h] = pos[h]
        col_idx[row_ptr[c[h]] + pos[h]] = c[h] + offs[s]
        pos += h
    return row_ptr, col_idx, slot


# ----------------------------------------------------------------- linearise
def linearize(spec, u_new, flag_new, u_old, flag_old, dt, mode="unew", lam=None, p_bh=None, controls=None,
              up_flip=None):
    """Residual and Jacobian of one backward-Euler step.

    mode="unew": derivatives with respect to the new state only (the Jacobian).
    mode="all": per-cell local variables are (u_new[nv], u_old[nv], ln k, phi);
    with ``lam`` (N, nb) given, the vector-Jacobian products
    lam^T dR/d(u_new, u_old, ln k, phi) are returned too.

    With ``p_bh`` (one value per well) the bottom-hole pressures are unknowns
    too, and every well gets an equation (the "w" rows and columns of the
    global Jacobian, Sec. 3.4.1): ``controls`` holds one (mode, phase, target)
    per well -- mode 0 fixes the bottom-hole pressure, R_w = p_bh - target;
    mode 1 fixes the surface rate of component ``phase``, R_w = s sum_perf
    q_phase - target with s = -1 for producers (production counted positive)
    and +1 for injectors.  Without ``controls`` every well is mode 0 at its own
    p_bh.  The extra outputs are ``well_res`` (nwell), ``well_B`` (nperf, nb)
    = dR_cell/dp_bh, ``well_C`` (nperf, nb) = dR_w/du_cell, ``well_D`` (nwell)
    = dR_w/dp_bh, each with its magnitude scale, perforations in well order.

    ``up_flip`` maps (direction, phase letter) to a boolean array over that
    direction's faces (``face_pairs`` order): where True, the upwind cell of
    that phase is the other one.  It exists for faces whose potential
    difference is zero to within rounding (a hydrostatic state): there the
    sign, and with it the side that reading X10 picks, is decided by rounding
    alone, the flux vanishes either way, and both one-sided derivatives are
    correct results.  Default: no face flipped.  ``face_dphi`` and
    ``face_dphi_mag`` hold every face's potential difference and its
    magnitude scale, the latter bounding how far rounding can move it.
    """
    nx, ny, nz = dims(spec)
    N = nx * ny * nz
    nv = nb = int(spec.nphase)
    L = nv if mode == "unew" else 2 * nv + 2
    # complex states give complex results (complex-step checks); real ones float64
    cdt = np.result_type(np.asarray(u_new), np.asarray(u_old), np.asarray(spec.lnk), np.asarray(spec.phi),
                         np.float64)
    u_new = np.asarray(u_new, dtype=cdt).reshape(nv, N)
    u_old = np.asarray(u_old, dtype=cdt).reshape(nv, N)
    lnk_v = np.asarray(spec.lnk, dtype=cdt)
    phi_v = np.asarray(spec.phi, dtype=cdt)

    un = [D.seed(u_new[v], L, v) for v in range(nv)]
    if mode == "all":
        uo = [D.seed(u_old[v], L, nv + v) for v in range(nv)]
        lnk = D.seed(lnk_v, L, 2 * nv)
        phi = D.seed(phi_v, L, 2 * nv + 1)
    else:
        uo = [D.const(u_old[v], N, L) for v in range(nv)]
        lnk = D.const(lnk_v, N, L)
        phi = D.const(phi_v, N, L)

    x_new = un[2] if nv == 3 else None
    x_old = uo[2] if nv == 3 else None
    pn = cell_properties(spec, un[0], un[1], x_new, flag_new, phi)
    po = cell_properties(spec, uo[0], uo[1], x_old, flag_old, phi)

    # ---- accumulation (ACCU): pore volume change of each component over dt
    vol = spec.dx * spec.dy * spec.dz
    mn, mo = masses(spec, pn), masses(spec, po)
    acc = [(mn[e] - mo[e]) * (vol / RB_FT3) / dt for e in range(nb)]

    R = np.zeros((N, nb), dtype=cdt)
    Rm = np.zeros((N, nb))
    row_ptr, col_idx, slot = bsr_pattern(spec)
    val = np.zeros((len(col_idx), nb, nb), dtype=cdt)
    valm = np.zeros((len(col_idx), nb, nb))
    gw = np.zeros((N, L), dtype=cdt) if lam is not None else None
    gwm = np.zeros((N, L)) if lam is not None else None
    alam = np.abs(lam) if lam is not None else None
    cells = np.arange(N)
    diag = row_ptr[:-1] + slot[3]

    def add_rows(rows, e, q: D, sign):
        np.add.at(R[:, e], rows, sign * q.v)
        np.add.at(Rm[:, e], rows, q.m)

    def add_block(blk_idx, e, gpart, gmpart, sign):
        np.add.at(val[:, e, :], blk_idx, sign * gpart)
        np.add.at(valm[:, e, :], blk_idx, gmpart)

    for e in range(nb):
        add_rows(cells, e, acc[e], 1.0)
        add_block(diag, e, acc[e].g[:, :nv], acc[e].gm[:, :nv], 1.0)
        if gw is not None:
            gw += lam[:, e:e + 1] * acc[e].g
            gwm += alam[:, e:e + 1] * acc[e].gm

    # ---- connection fluxes (BulkConn): two-point, phase-upwinded
    z = depth(spec)
    phases = ["w", "o", "g"][:nb]
    face_flux = np.zeros((3, nb, N), dtype=cdt)
    face_flux_mag = np.zeros((3, nb, N))
    face_dphi = {}
    face_dphi_mag = {}
    for d in range(3):
        fi, fj = face_pairs(spec, d)
        if len(fi) == 0:
            continue
        K2 = 2 * L
        Pi = {key: val_.take(fi).embed(K2, 0) for key, val_ in pn.items() if val_ is not None}
        Pj = {key: val_.take(fj).embed(K2, L) for key, val_ in pn.items() if val_ is not None}
        T = transmissibility(spec, d, lnk.take(fi).embed(K2, 0), lnk.take(fj).embed(K2, L))
        dz_ij = z[fi] - z[fj]
        F = {}
        for a in phases:
            gamma = (Pi["rho_" + a] + Pj["rho_" + a]) * (0.5 * GRAV)
            dphi = (Pi["p_" + a] - Pj["p_" + a]) - gamma * dz_ij
            up_i = dphi.v >= 0.0
            if up_flip is not None and (d, a) in up_flip:
                up_i = up_i ^ np.asarray(up_flip[(d, a)], dtype=bool)
            lam_up = where(up_i, Pi["lam_" + a], Pj["lam_" + a])
            F[a] = T * lam_up * dphi
            F["up_" + a] = up_i
            face_dphi[(d, a)] = dphi.v
            face_dphi_mag[(d, a)] = dphi.m
        comp = [F["w"], F["o"]]
        if nb == 3:
            rs_up = where(F["up_o"], Pi["Rs"], Pj["Rs"])
            comp.append(F["g"] + rs_up * F["o"])
        s_plus = slot[4 + d]    # +x, +y, +z neighbour slots
        s_minus = slot[2 - d]   # -x, -y, -z neighbour slots
        blk_ii = diag[fi]
        blk_ij = row_ptr[fi] + s_plus[fi]
        blk_ji = row_ptr[fj] + s_minus[fj]
        blk_jj = diag[fj]
        for e in range(nb):
            q = comp[e]
            face_flux[d, e, fi] = q.v
            face_flux_mag[d, e, fi] = q.m
            add_rows(fi, e, q, 1.0)
            add_rows(fj, e, q, -1.0)
            gi, gj = q.g[:, :nv], q.g[:, L:L + nv]
            gmi, gmj = q.gm[:, :nv], q.gm[:, L:L + nv]
            add_block(blk_ii, e, gi, gmi, 1.0)
            add_block(blk_ij, e, gj, gmj, 1.0)
            add_block(blk_ji, e, gi, gmi, -1.0)
            add_block(blk_jj, e, gj, gmj, -1.0)
            if gw is not None:
                w = (lam[fi, e] - lam[fj, e])[:, None]
                np.add.at(gw, fi, w * q.g[:, :L])
                np.add.at(gw, fj, w * q.g[:, L:])
                wm = (alam[fi, e] + alam[fj, e])[:, None]
                np.add.at(gwm, fi, wm * q.gm[:, :L])
                np.add.at(gwm, fj, wm * q.gm[:, L:])

    # ---- wells (AllWells): perforation sources at the bottom-hole pressure
    nwell = len(spec.wells)
    unknown_bhp = p_bh is not None
    Lw = L + 1 if unknown_bhp else L      # slot L: the well's own p_bh
    if unknown_bhp:
        p_bh = np.asarray(p_bh, dtype=np.float64)
        if controls is None:
            controls = [(0, 0, float(w.p_bh)) for w in spec.wells]
        w_res = np.zeros(nwell, dtype=cdt)
        w_res_m = np.zeros(nwell)
        w_D = np.zeros(nwell, dtype=cdt)
        w_D_m = np.zeros(nwell)
        w_B, w_B_m, w_C, w_C_m = [], [], [], []
    well_q = np.zeros((N, nb), dtype=cdt)
    well_rate = np.zeros((nwell, nb), dtype=cdt)
    well_grad = []          # per well: (cells, dq/dlocal of shape (nperf, nb, L))
    for iw, w in enumerate(spec.wells):
        cells_w = np.asarray(w.cells, dtype=np.int64)
        n_w = len(cells_w)
        if n_w == 0:
            well_grad.append((cells_w, np.zeros((0, nb, L))))
            if unknown_bhp:
                mode, _, target = controls[iw]
                w_res[iw] = (p_bh[iw] - target) if mode == 0 else -target
                w_res_m[iw] = (abs(p_bh[iw]) + abs(target)) if mode == 0 else abs(target)
                w_D[iw] = 1.0 if mode == 0 else 0.0
                w_D_m[iw] = abs(w_D[iw])
            continue
        P = {key: val_.take(cells_w).embed(Lw, 0) for key, val_ in pn.items() if val_ is not None}
        WI = well_index(spec, w, lnk.take(cells_w)).embed(Lw, 0)
        zero = D.const(0.0, n_w, Lw)
        pw = D.seed(np.full(n_w, p_bh[iw]), Lw, L) if unknown_bhp else w.p_bh
        if w.kind == 0:  # producer: every mobile phase leaves where p > p_bh
            drive = P["p_o"] - pw
            open_ = drive.v > 0.0
            qs = [where(open_, WI * P["lam_" + a] * (pw - P["p_o"]), zero) for a in phases]
            if nb == 3:
                qs[2] = qs[2] + P["Rs"] * qs[1]
        else:  # injector of one phase with the cell's total mobility
            drive = pw - P["p_o"]
            open_ = drive.v > 0.0
            mob = P["kr_w"] * P["imu_w"] + P["kr_o"] * P["imu_o"]
            if nb == 3:
                mob = mob + P["kr_g"] * P["imu_g"]
            b_inj = P["b_w"] if w.phase == 0 else P["b_g"]
            q_inj = where(open_, WI * mob * b_inj * drive, zero)
            qs = [zero if e != (0 if w.phase == 0 else 2) else q_inj for e in range(nb)]
        well_grad.append((cells_w, np.stack([qs[e].g[:, :L] for e in range(nb)], axis=1)))
        for e in range(nb):
            q = qs[e]
            well_rate[iw, e] = q.v.sum()
            well_q[cells_w, e] += q.v
            add_rows(cells_w, e, q, -1.0)
            add_block(diag[cells_w], e, q.g[:, :nv], q.gm[:, :nv], -1.0)
            if gw is not None:
                np.add.at(gw, cells_w, -lam[cells_w, e:e + 1] * q.g[:, :L])
                np.add.at(gwm, cells_w, alam[cells_w, e:e + 1] * q.gm[:, :L])
        if unknown_bhp:
            # the cell rows' dependence on p_bh (R_cell holds -q)
            w_B.append(np.stack([-qs[e].g[:, L] for e in range(nb)], axis=1))
            w_B_m.append(np.stack([qs[e].gm[:, L] for e in range(nb)], axis=1))
            mode, ph, target = controls[iw]
            if mode == 0:
                w_res[iw] = p_bh[iw] - target
                w_res_m[iw] = abs(p_bh[iw]) + abs(target)
                w_D[iw] = 1.0
                w_D_m[iw] = 1.0
                w_C.append(np.zeros((n_w, nb), dtype=cdt))
                w_C_m.append(np.zeros((n_w, nb)))
            else:
                sgn = -1.0 if w.kind == 0 else 1.0
                q = qs[ph]
                w_res[iw] = sgn * q.v.sum() - target
                w_res_m[iw] = q.m.sum() + abs(target)
                w_D[iw] = sgn * q.g[:, L].sum()
                w_D_m[iw] = q.gm[:, L].sum()
                c_blk = np.zeros((n_w, nb), dtype=cdt)
                c_blk[:, :nv] = sgn * q.g[:, :nv]
                c_mag = np.zeros((n_w, nb))
                c_mag[:, :nv] = q.gm[:, :nv]
                w_C.append(c_blk)
                w_C_m.append(c_mag)

    out = {
        "R": R, "R_mag": Rm, "row_ptr": row_ptr, "col_idx": col_idx,
        "val": val, "val_mag": valm, "acc": np.stack([a.v for a in acc], axis=1),
        "well_q": well_q, "well_rate": well_rate, "well_grad": well_grad,
        "face_flux": face_flux, "face_flux_mag": face_flux_mag,
        "face_dphi": face_dphi, "face_dphi_mag": face_dphi_mag,
    }
    if unknown_bhp:
        cat = lambda parts: np.concatenate(parts) if parts else np.zeros((0, nb))
        out.update(well_res=w_res, well_res_mag=w_res_m, well_D=w_D, well_D_mag=w_D_m,
                   well_B=cat(w_B), well_B_mag=cat(w_B_m), well_C=cat(w_C), well_C_mag=cat(w_C_m))
    if gw is not None:
        out["g_unew"] = gw[:, :nv].T.copy()
        out["g_uold"] = gw[:, nv:2 * nv].T.copy()
        out["g_lnk"] = gw[:, 2 * nv].copy()
        out["g_phi"] = gw[:, 2 * nv + 1].copy()
        out["g_unew_mag"] = gwm[:, :nv].T.copy()
        out["g_uold_mag"] = gwm[:, nv:2 * nv].T.copy()
        out["g_lnk_mag"] = gwm[:, 2 * nv].copy()
        out["g_phi_mag"] = gwm[:, 2 * nv + 1].copy()
    return out
