"""Buckley-Leverett pin of the oracle (1-D, two-phase, incompressible).

With b = 1, no compressibility, no gravity, no capillary pressure, S_wc =
S_or = 0 and Corey exponents 2 (k_rw = S^2, k_ro = (1-S)^2), the fractional
flow is f(S) = S^2 / (S^2 + r (1-S)^2) with r = mu_w / mu_o.  Injecting water
into oil gives a shock at the Welge tangent point, which for exponent 2 has
the closed form S_f = sqrt(r / (1 + r)); behind it each saturation S travels
to x = (Q / (phi A)) f'(S), where Q is the cumulative injected volume (the
solution is self-similar in Q, so a varying injection rate does not matter).
The oracle's Newton time stepping must converge to this solution as the grid
is refined.
"""
import math

import numpy as np
import pytest

from oracle.blackoil import RB_FT3
from oracle.newton import newton_step
from paper_2406_10862_gb300 import workloads as W

R_VISC = 0.5   # mu_w / mu_o


def bl_grid(n, length=1000.0):
    t = W.synthetic_tables()
    m = len(t["tab_p"])
    g = W.make_grid(n, 1, 1, np.full(n, math.log(100.0)), np.full(n, 0.2), [], nphase=2,
                    dx=length / n, dy=10.0, dz=10.0,
                    tab_Bo=np.ones(m), tab_muo=np.full(m, 1.0), cw=0.0, cr=0.0, bw_ref=1.0,
                    muw=R_VISC, swc=0.0, sorw=0.0, krw_max=1.0, kro_cw=1.0, pcow_max=0.0)
    g.wells = [W.Well(kind=1, phase=0, p_bh=1100.0, cells=np.array([0])),
               W.Well(kind=0, phase=0, p_bh=900.0, cells=np.array([n - 1]))]
    return g


def bl_exact(xd, qd):
    """Analytic S_w at dimensionless positions xd after qd injected pore
    volumes."""
    sf = math.sqrt(R_VISC / (1.0 + R_VISC))
    s = np.linspace(1.0, sf, 20001)
    dfds = 2 * s * R_VISC * (1 - s) / (s * s + R_VISC * (1 - s) ** 2) ** 2
    x_of_s = qd * dfds                                 # increasing from 0 at S=1 to x_f at S_f
    out = np.interp(xd, x_of_s, s, right=0.0)
    return out, qd * dfds[-1]


def run_bl(n, target_pv=0.35, steps=120):
    g = bl_grid(n)
    pv = 0.2 * 1000.0 * 10.0 * 10.0                    # ft^3
    u = np.zeros((2, n))
    u[0] = 1000.0
    u[1] = 0.0
    flag = np.zeros(n, dtype=np.int8)
    injected = 0.0                                      # ft^3 of water
    dt = 0.01
    for _ in range(4 * steps):
        u_new, flag, o, _ = newton_step(g, u, flag, dt)
        q_inj = o["well_q"][0, 0]                       # stb/day = rb/day with b = 1
        injected += q_inj * dt * RB_FT3
        u = u_new
        remaining = target_pv * pv - injected
        if remaining <= 1e-9 * pv:
            break
        dt = min(remaining, target_pv * pv / steps) / (q_inj * RB_FT3)
    return g, u, injected / pv


@pytest.mark.slow
def test_buckley_leverett_convergence():
    sf = math.sqrt(R_VISC / (1 + R_VISC))
    errs, fronts = [], []
    for n in (100, 200, 400):
        g, u, qd = run_bl(n)
        assert qd == pytest.approx(0.35, rel=1e-4)
        xd = (np.arange(n) + 0.5) / n
        exact, xf = bl_exact(xd, qd)
        errs.append(np.mean(np.abs(u[1] - exact)))
        # the numerical front (where S_w crosses S_f / 2) against the shock
        front = xd[np.argmax(u[1] < 0.5 * sf)]
        fronts.append(abs(front - xf))
        # no water ahead of the smeared shock
        assert np.all(u[1][xd > xf + 0.1] < 1e-3)
    assert errs[1] < errs[0] and errs[2] < errs[1]
    assert fronts[2] < fronts[0] and fronts[2] < 0.03
    assert errs[2] < 0.02
