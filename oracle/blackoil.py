"""Cell properties of the black-oil model, written out plainly (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The paper states the black-oil closure only in general terms: in the black-oil
model the phase saturations, the phase compositions and the phase molar
densities follow explicitly from pressure and the component amounts (Sec. 2.1,
after the constraint equations), and the PVT, SAT and ROCK modules compute
fluid, saturation and rock properties per cell (Sec. 3.2.3).  The concrete
textbook model below (table interpolation, Corey curves, Stone's second model,
capillary pressure, rock compressibility) is this library's reading of those
modules; every choice is listed with its reason in the design notes.

Variables per cell (natural variables, block order p, S_w, X):
* three-phase: ``X = S_g`` where the flag is 0 (saturated: free gas may
  exist), ``X = R_s`` where the flag is 1 (undersaturated: no free gas);
* two-phase oil-water: ``(p, S_w)`` only.

Units are oil-field units: psi, ft, mD, cP, day, stb, scf, rb, lb/ft^3.
"""
from __future__ import annotations

import numpy as np

from .dual import D, where

RB_FT3 = 5.614583        # ft^3 per reservoir barrel
C_DARCY = 0.001127       # rb cP / (day psi mD ft)
GRAV = 1.0 / 144.0       # psi per (lb/ft^3 * ft)


# --------------------------------------------------------------------- tables
def table_columns(spec):
    """The interpolated columns: reciprocal formation volume factors and
    reciprocal viscosities, plus the solution gas-oil ratio, all versus p.
    Interpolating 1/B and 1/mu (not B and mu) is a reading of a silent paper."""
    p = np.asarray(spec.tab_p, dtype=np.float64)
    cols = {
        "b_o": 1.0 / np.asarray(spec.tab_Bo, dtype=np.float64),
        "imu_o": 1.0 / np.asarray(spec.tab_muo, dtype=np.float64),
        "b_g": 1.0 / np.asarray(spec.tab_Bg, dtype=np.float64),
        "imu_g": 1.0 / np.asarray(spec.tab_mug, dtype=np.float64),
        "Rs": np.asarray(spec.tab_Rs, dtype=np.float64),
    }
    return p, cols


def segment(knots, x):
    """Index k of the linear piece used at x: the largest k <= nrow-2 with
    knots[k] <= x (so a value on a knot takes the piece to its right, and the
    end pieces extend linearly beyond the table)."""
    nseg = len(knots) - 1
    k = np.zeros(np.shape(x), dtype=np.int64)
    for i in range(1, nseg):
        k = np.where(x >= knots[i], i, k)
    return k


def interp_on(knots, y, k, x: D) -> D:
    """Linear piece number k of the table (knots, y), evaluated at x."""
    slope = (y[k + 1] - y[k]) / (knots[k + 1] - knots[k])
    return (x - knots[k]) * slope + y[k]


def interp(knots, y, x: D) -> D:
    return interp_on(knots, y, segment(knots, x.v), x)


# ------------------------------------------------------------------ saturation
def clamp01(s: D) -> D:
    """Clamp to [0, 1]; outside the interval the derivative is zero, on the
    interval's ends the interior formula is kept."""
    zero = D.const(0.0, s.n, s.k)
    one = D.const(1.0, s.n, s.k)
    return where(s.v < 0.0, zero, where(s.v > 1.0, one, s))


def corey(s_norm: D, kmax, expo) -> D:
    return kmax * (s_norm ** expo)


def relperm(spec, sw: D, sg: D | None):
    """Corey curves and, with three phases, Stone's second model for oil.

    Returns (kr_w, kr_o, kr_g, s_w_norm, s_g_norm); kr_g and s_g_norm are None
    with two phases."""
    swc, sorw = spec.swc, spec.sorw
    s_w = clamp01((sw - swc) / (1.0 - swc - sorw))
    s_ow = clamp01((1.0 - sw - sorw) / (1.0 - swc - sorw))
    kr_w = corey(s_w, spec.krw_max, spec.nw)
    kr_ow = corey(s_ow, spec.kro_cw, spec.now)
    if sg is None:
        return kr_w, kr_ow, None, s_w, None
    sgc, sorg = spec.sgc, spec.sorg
    s_g = clamp01((sg - sgc) / (1.0 - swc - sgc - sorg))
    s_og = clamp01((1.0 - sg - swc - sorg) / (1.0 - swc - sorg))
    kr_g = corey(s_g, spec.krg_max, spec.ng)
    kr_og = corey(s_og, spec.kro_cw, spec.nog)
    kc = spec.kro_cw
    # Stone II in the normalised form of Aziz and Settari, floored at zero.
    kr_o = kc * ((kr_ow / kc + kr_w) * (kr_og / kc + kr_g) - (kr_w + kr_g))
    kr_o = where(kr_o.v < 0.0, D.const(0.0, kr_o.n, kr_o.k), kr_o)
    return kr_w, kr_o, kr_g, s_w, s_g


# ------------------------------------------------------------------ properties
def cell_properties(spec, p: D, sw: D, x: D | None, flag, phi_ref):
    """All per-cell quantities the residual needs, as dual numbers.

    ``x`` is the third unknown (S_g or R_s by ``flag``) with three phases and
    None with two; ``phi_ref`` is the reference porosity of the same cells (an
    array, or a dual number when its derivative is wanted).  The returned dict
    holds (phase letters w, o, g):
    b_*, imu_*, Rs, phi, S_*, kr_*, p_* (phase pressures), rho_*, lam_*.
    """
    n, k = p.n, p.k
    three = spec.nphase == 3
    knots, cols = table_columns(spec)
    out = {}

    # water: linear compressibility, constant viscosity
    b_w = (1.0 + spec.cw * (p - spec.p_ref)) * spec.bw_ref
    out["b_w"], out["imu_w"] = b_w, D.const(1.0 / spec.muw, n, k)

    # rock
    out["phi"] = (1.0 + spec.cr * (p - spec.p_ref)) * phi_ref

    if three:
        flag = np.asarray(flag)
        unsat = flag == 1
        # saturated branch: table values at p
        kp = segment(knots, p.v)
        b_o_sat = interp_on(knots, cols["b_o"], kp, p)
        imu_o_sat = interp_on(knots, cols["imu_o"], kp, p)
        rs_sat = interp_on(knots, cols["Rs"], kp, p)
        # undersaturated branch: bubble point from the inverse of R_s(p), then
        # a constant oil compressibility and viscosibility above it.  The
        # table piece used at p_b is the piece the given R_s falls in.
        # (evaluated for every cell and then selected by the flag; a flat R_s
        # column makes the unselected branch infinite, which is harmless)
        with np.errstate(all="ignore"):
            kr = segment(cols["Rs"], x.v)
            pb = interp_on(cols["Rs"], knots, kr, x)
            dp = p - pb
            b_o_un = interp_on(knots, cols["b_o"], kr, pb) * (1.0 + spec.co_under * dp)
            imu_o_un = interp_on(knots, cols["imu_o"], kr, pb) * (1.0 - spec.cmu_under * dp)
        out["b_o"] = where(unsat, b_o_un, b_o_sat)
        out["imu_o"] = where(unsat, imu_o_un, imu_o_sat)
        out["Rs"] = where(unsat, x, rs_sat)
        sg = where(unsat, D.const(0.0, n, k), x)
        out["b_g"] = interp(knots, cols["b_g"], p)
        out["imu_g"] = interp(knots, cols["imu_g"], p)
    else:
        out["b_o"] = interp(knots, cols["b_o"], p)
        out["imu_o"] = interp(knots, cols["imu_o"], p)
        out["Rs"] = D.const(0.0, n, k)
        sg = None

    out["S_w"] = sw
    out["S_g"] = sg
    out["S_o"] = (1.0 - sw - sg) if three else (1.0 - sw)

    kr_w, kr_o, kr_g, s_w, s_g = relperm(spec, sw, sg)
    out["kr_w"], out["kr_o"], out["kr_g"] = kr_w, kr_o, kr_g

    # capillary pressures and phase pressures (oil pressure is primary)
    pc_ow = ((1.0 - s_w) ** 2.0) * spec.pcow_max
    out["p_o"] = p
    out["p_w"] = p - pc_ow
    if three:
        pc_go = (s_g ** 2.0) * spec.pcgo_max
        out["p_g"] = p + pc_go

    # mass densities at reservoir conditions
    out["rho_w"] = out["b_w"] * spec.rho_wsc
    out["rho_o"] = (out["Rs"] * spec.rho_gsc / RB_FT3 + spec.rho_osc) * out["b_o"]
    if three:
        out["rho_g"] = out["b_g"] * spec.rho_gsc / RB_FT3

    # mobilities in surface volume per reservoir volume per cP
    out["lam_w"] = kr_w * (out["b_w"] * out["imu_w"])
    out["lam_o"] = kr_o * (out["b_o"] * out["imu_o"])
    if three:
        out["lam_g"] = kr_g * (out["b_g"] * out["imu_g"])
    return out


def masses(spec, pr):
    """Component amounts per unit bulk volume, phi * S * b, in surface volume
    per reservoir volume (eq. 4 specialised to black oil, where the gas
    component is both free and dissolved in oil through R_s)."""
    m_w = pr["phi"] * pr["S_w"] * pr["b_w"]
    m_o = pr["phi"] * pr["S_o"] * pr["b_o"]
    if spec.nphase == 2:
        return [m_w, m_o]
    m_g = pr["phi"] * (pr["S_g"] * pr["b_g"] + pr["Rs"] * pr["S_o"] * pr["b_o"])
    return [m_w, m_o, m_g]
