"""Seeded synthetic inputs: grids, rock, fluid tables, wells and states.

This module only *draws* inputs (numpy ``default_rng`` with fixed seeds); it
contains none of the linearisation's arithmetic, so both the CUDA path and the
CPU checker can be fed from it without sharing any of the method.

The workloads have the shapes of the paper's black-oil cases but none of their
data: a 10x10x3 three-phase box with a gas injector and a producer in opposite
corners (the shape of SPE1), a layered 100x100x20 box with five wells, a
channelised 60x220x85 oil-water model (the shape of SPE10 model 2), an
ensemble of 64 uneven boxes, and a 100x100x10 history-matching case.  Every
value (tables, permeability fields, end points) is synthetic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Well:
    kind: int            # 0 producer, 1 injector
    phase: int           # injected phase for injectors: 0 water, 2 gas
    p_bh: float          # bottom-hole pressure, psi
    cells: np.ndarray    # perforated cells (natural index), int64
    rw: float = 0.25     # wellbore radius, ft
    skin: float = 0.0


@dataclasses.dataclass
class GridDesc:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    top_depth: float
    nphase: int
    lnk: np.ndarray      # ln(k_x / mD), N
    phi: np.ndarray      # reference porosity, N
    kz_over_kx: float
    cr: float
    p_ref: float
    tab_p: np.ndarray
    tab_Bo: np.ndarray
    tab_Bg: np.ndarray
    tab_Rs: np.ndarray
    tab_muo: np.ndarray
    tab_mug: np.ndarray
    bw_ref: float
    cw: float
    muw: float
    rho_osc: float
    rho_gsc: float
    rho_wsc: float
    co_under: float
    cmu_under: float
    swc: float
    sorw: float
    sorg: float
    sgc: float
    nw: float
    now: float
    ng: float
    nog: float
    krw_max: float
    krg_max: float
    kro_cw: float
    pcow_max: float
    pcgo_max: float
    wells: list

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def cell(self, i, j, k) -> int:
        return i + self.nx * (j + self.ny * k)

    def column(self, i, j) -> np.ndarray:
        return np.array([self.cell(i, j, k) for k in range(self.nz)], dtype=np.int64)


@dataclasses.dataclass
class State:
    u_new: np.ndarray    # (nv, N) float64, variable-major
    flag_new: np.ndarray  # (N,) int8
    u_old: np.ndarray
    flag_old: np.ndarray
    dt: float


# ----------------------------------------------------------------- the fluid
def synthetic_tables(nrow=20, p_lo=400.0, p_hi=6400.0):
    """Monotone synthetic PVT rows (not from any benchmark deck):
    Rs = 0.3 p, Bo = 1 + 1.2e-4 Rs, Bg = 5/p, mu_o = 1.2 - 1e-4 p,
    mu_g = 0.012 + 3e-6 p."""
    p = np.linspace(p_lo, p_hi, nrow)
    rs = 0.3 * p
    return dict(tab_p=p, tab_Rs=rs, tab_Bo=1.0 + 1.2e-4 * rs, tab_Bg=5.0 / p,
                tab_muo=1.2 - 1.0e-4 * p, tab_mug=0.012 + 3.0e-6 * p)


def default_fluid():
    return dict(
        kz_over_kx=0.1, cr=4e-6, p_ref=4800.0,
        bw_ref=1.0, cw=3e-6, muw=0.5,
        rho_osc=50.0, rho_gsc=0.06, rho_wsc=62.4,
        co_under=1e-5, cmu_under=0.0,
        swc=0.12, sorw=0.20, sorg=0.10, sgc=0.0,
        nw=2.0, now=2.0, ng=2.0, nog=2.0,
        krw_max=0.4, krg_max=0.9, kro_cw=1.0,
        pcow_max=4.0, pcgo_max=2.0,
        **synthetic_tables(),
    )


def make_grid(nx, ny, nz, lnk, phi, wells, nphase=3, dx=300.0, dy=300.0, dz=30.0,
              top_depth=8000.0, **over):
    f = default_fluid()
    f.update(over)
    return GridDesc(nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, top_depth=top_depth,
                    nphase=nphase, lnk=np.ascontiguousarray(lnk, dtype=np.float64),
                    phi=np.ascontiguousarray(phi, dtype=np.float64), wells=wells, **f)


# ----------------------------------------------------------------- states
def perturbed_state(g: GridDesc, rng, p0=4800.0, sw0=0.12, dt=1.0, frac_unsat=0.0,
                    dp_sd=20.0, ds_hi=0.02, rs_hi=0.9):
    """Old state uniform (p0, sw0, S_g = 0, saturated); new state the old one
    plus a seeded perturbation, so that every flux and derivative is
    non-trivial.  A fraction ``frac_unsat`` of cells is flagged
    undersaturated in both states, with X = R_s drawn as U(0.3, rs_hi) times
    the table's largest R_s (rs_hi = 0.7 keeps it below the saturated R_s of
    the table at p0 = 4800 psi, a consistent undersaturated oil)."""
    N, nv = g.N, g.nphase
    u_old = np.zeros((nv, N))
    u_old[0] = p0
    u_old[1] = sw0
    flag = np.zeros(N, dtype=np.int8)
    if nv == 3 and frac_unsat > 0.0:
        unsat = rng.random(N) < frac_unsat
        flag[unsat] = 1
        rs_max = float(np.max(g.tab_Rs))
        u_old[2, unsat] = rng.uniform(0.3, rs_hi, unsat.sum()) * rs_max
    u_new = u_old.copy()
    u_new[0] += rng.normal(0.0, dp_sd, N)
    u_new[1] += rng.uniform(0.0, ds_hi, N)
    if nv == 3:
        sat = flag == 0
        u_new[2, sat] += rng.uniform(0.0, ds_hi, sat.sum())
        un = flag == 1
        u_new[2, un] *= rng.uniform(0.97, 1.03, un.sum())
    return State(u_new=u_new, flag_new=flag.copy(), u_old=u_old, flag_old=flag.copy(), dt=dt)


# ----------------------------------------------------------------- workloads
def spe1_like(seed=1):
    """10x10x3 three-phase box (300 cells, dx=dy=300 ft, dz=30 ft), ln k ~
    N(ln 100, 1) i.i.d., phi ~ U(0.15, 0.3), gas injector in cell (0,0,0) at
    5500 psi, producer in cell (9,9,2) at 4000 psi, p=4800, S_w=0.12, S_g=0,
    dt = 1 day."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = 10, 10, 3
    N = nx * ny * nz
    lnk = rng.normal(math.log(100.0), 1.0, N)
    phi = rng.uniform(0.15, 0.3, N)
    wells = [Well(kind=1, phase=2, p_bh=5500.0, cells=np.array([0], dtype=np.int64)),
             Well(kind=0, phase=0, p_bh=4000.0, cells=np.array([9 + 10 * (9 + 10 * 2)], dtype=np.int64))]
    g = make_grid(nx, ny, nz, lnk, phi, wells)
    return g, perturbed_state(g, rng)


def layered_lnk(rng, nx, ny, nz, lo=10.0, hi=1000.0, noise=0.5):
    means = rng.uniform(math.log(lo), math.log(hi), nz)
    return (np.repeat(means, nx * ny) + rng.normal(0.0, noise, nx * ny * nz))


def layered_box(seed=2, nx=100, ny=100, nz=20, frac_unsat=0.0):
    """100x100x20 three-phase box (200 000 cells): layered ln k (per-layer mean
    ~ U(ln 10, ln 1000) mD plus N(0, 0.5) noise), kz/kx = 0.1, producers at
    3500 psi in columns (4,4), (95,4), (4,95), (95,95) and a gas injector at
    5500 psi in column (49,49), all layers perforated."""
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    lnk = layered_lnk(rng, nx, ny, nz)
    phi = rng.uniform(0.15, 0.3, N)
    g = make_grid(nx, ny, nz, lnk, phi, [])
    cx, cy = nx // 2 - 1, ny // 2 - 1
    lo_x, hi_x, lo_y, hi_y = min(4, nx - 1), max(nx - 5, 0), min(4, ny - 1), max(ny - 5, 0)
    g.wells = [Well(kind=0, phase=0, p_bh=3500.0, cells=g.column(i, j))
               for (i, j) in [(lo_x, lo_y), (hi_x, lo_y), (lo_x, hi_y), (hi_x, hi_y)]]
    g.wells.append(Well(kind=1, phase=2, p_bh=5500.0, cells=g.column(cx, cy)))
    return g, perturbed_state(g, rng, frac_unsat=frac_unsat)


def channelised_ow(seed=3, nx=60, ny=220, nz=85, n_channels=12):
    """Two-phase oil-water model with the shape of SPE10 model 2 (60x220x85,
    1 122 000 cells, dx=dy=50 ft, dz=5 ft): a low-permeability background
    (median 1 mD) crossed by seeded sinuous high-permeability channels
    (median 1000 mD), porosity correlated with ln k, five-spot wells (water
    injector at 8000 psi in the centre, producers at 4000 psi in the corners),
    p=6000 psi, S_w = S_wc = 0.2."""
    rng = np.random.default_rng(seed)
    lnk = rng.normal(math.log(1.0), 1.0, (nz, ny, nx))
    xs = np.arange(nx)[None, :]
    ys = np.arange(ny)[:, None]
    for _ in range(n_channels):
        amp = rng.uniform(5, 20)
        lam = rng.uniform(40, 120)
        psi = rng.uniform(0, 2 * math.pi)
        y0 = rng.uniform(0, ny)
        width = rng.uniform(3, 8)
        k0 = int(rng.integers(0, nz))
        k1 = min(nz, k0 + int(rng.integers(4, 11)))
        # channel meanders along y; its centreline in x varies with y
        xc = (nx / 2.0 + (y0 - ny / 2.0) * nx / ny) + amp * np.sin(2 * math.pi * ys / lam + psi)
        inside = np.abs(xs - xc) < width / 2.0
        for k in range(k0, k1):
            draw = rng.normal(math.log(1000.0), 0.5, (ny, nx))
            lnk[k][inside] = draw[inside]
    lnk = lnk.ravel()
    phi = np.clip(0.12 + 0.02 * (lnk - math.log(10.0)), 0.05, 0.35)
    g = make_grid(nx, ny, nz, lnk, phi, [], nphase=2, dx=50.0, dy=50.0, dz=5.0, swc=0.2)
    g.wells = [Well(kind=1, phase=0, p_bh=8000.0, cells=g.column(nx // 2, ny // 2))]
    for (i, j) in [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1)]:
        g.wells.append(Well(kind=0, phase=0, p_bh=4000.0, cells=g.column(i, j)))
    return g, perturbed_state(g, rng, p0=6000.0, sw0=0.2)


def ensemble(n_models=64, seed=4, lo=2e4, hi=4e5):
    """64 three-phase boxes with cell counts log-uniform in [2e4, 4e5]: nz = 10,
    nx = round(sqrt(N/10)), ny = round(N/(10 nx)); each with its own ln k ~
    N(ln 100, 1.5) (seed 4000 + m), an injector and a producer in opposite
    corner columns; the physics of the 10x10x3 case."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(n_models):
        target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        nz = 10
        nx = max(2, int(round(math.sqrt(target / nz))))
        ny = max(2, int(round(target / (nz * nx))))
        r = np.random.default_rng(4000 + m)
        N = nx * ny * nz
        lnk = r.normal(math.log(100.0), 1.5, N)
        phi = r.uniform(0.15, 0.3, N)
        g = make_grid(nx, ny, nz, lnk, phi, [])
        g.wells = [Well(kind=1, phase=2, p_bh=5500.0, cells=g.column(0, 0)),
                   Well(kind=0, phase=0, p_bh=4000.0, cells=g.column(nx - 1, ny - 1))]
        out.append((g, perturbed_state(g, r)))
    return out


def tiny(nx, ny, nz, nphase=3, seed=0, frac_unsat=0.3, wells=True, rs_hi=0.9, **over):
    """Small random grid for parity and edge-case tests: random ln k and phi,
    a producer and (three-phase: gas, two-phase: water) injector when the grid
    has at least two columns, mixed saturated/undersaturated cells."""
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    lnk = rng.normal(math.log(100.0), 1.0, N)
    phi = rng.uniform(0.15, 0.3, N)
    g = make_grid(nx, ny, nz, lnk, phi, [], nphase=nphase, **over)
    if wells:
        g.wells = [Well(kind=0, phase=0, p_bh=4600.0, cells=g.column(nx - 1, ny - 1))]
        if nx * ny > 1:
            g.wells.append(Well(kind=1, phase=2 if nphase == 3 else 0, p_bh=5100.0,
                                cells=g.column(0, 0)))
    return g, perturbed_state(g, rng, frac_unsat=frac_unsat if nphase == 3 else 0.0, rs_hi=rs_hi)


def history_match(nx=100, ny=100, nz=10, seed_truth=51, seed_prior=52, seed_rock=5, nsteps=20, dt=1.0):
    """History-matching case on a 100x100x10 three-phase box (100 000 cells):
    a truth ln k and a prior ln k, both layered (per-layer means ~ U(ln 10,
    ln 1000) mD plus N(0, 0.5) noise) from different seeds; porosity, wells
    (four producers at 3500 psi, a gas injector at 5500 psi, all layers) and
    the uniform initial state (p = 4800 psi, S_w = 0.12, S_g = 0) shared;
    20 steps of 1 day.  Returns (grid with the prior ln k, initial state,
    ln k truth, ln k prior, dt, number of steps)."""
    g, _ = layered_box(seed=seed_rock, nx=nx, ny=ny, nz=nz)
    lnk_truth = layered_lnk(np.random.default_rng(seed_truth), nx, ny, nz)
    lnk_prior = layered_lnk(np.random.default_rng(seed_prior), nx, ny, nz)
    g.lnk = np.ascontiguousarray(lnk_prior)
    N = g.N
    u0 = np.zeros((3, N))
    u0[0] = 4800.0
    u0[1] = 0.12
    f0 = np.zeros(N, dtype=np.int8)
    st = State(u_new=u0.copy(), flag_new=f0.copy(), u_old=u0, flag_old=f0, dt=dt)
    return g, st, lnk_truth, lnk_prior, dt, nsteps


# ----------------------------------------------------------------- moving fronts
def front_state(g: GridDesc, seed, fronts, width=1.5, ds_front=0.02, ds_bg=2e-3, frac_unsat=0.2, dt=1.0):
    """Pair of states whose saturations differ strongly only on thin moving
    fronts, as around the injectors of a gas/water alternating flood.

    ``fronts`` is a list of (ci, cj, ck, radius, phase) in cell units with
    phase 0 (water) or 2 (gas): the cells whose centre lies within ``width``
    of that sphere gain ``ds_front`` of that phase (gas only where the cell is
    saturated).  Every other cell moves by less than ``ds_bg`` per phase; a
    fraction ``frac_unsat`` of cells (three-phase) is undersaturated with X =
    R_s rescaled by up to 3 %.  Some cells switch between saturated and
    undersaturated over the step."""
    rng = np.random.default_rng(seed)
    N, nv = g.N, g.nphase
    c = np.arange(N)
    i, j, k = c % g.nx, (c // g.nx) % g.ny, c // (g.nx * g.ny)
    u_old = np.zeros((nv, N))
    u_old[0] = 4800.0 + rng.normal(0.0, 50.0, N)
    u_old[1] = 0.12 + rng.uniform(0.0, 0.2, N)
    f_old = np.zeros(N, dtype=np.int8)
    if nv == 3:
        u_old[2] = rng.uniform(0.0, 0.1, N)
        unsat = rng.random(N) < frac_unsat
        f_old[unsat] = 1
        u_old[2, unsat] = rng.uniform(0.3, 0.9, int(unsat.sum())) * float(np.max(g.tab_Rs))
    u_new = u_old.copy()
    f_new = f_old.copy()
    u_new[0] += rng.normal(0.0, 20.0, N)
    u_new[1] += rng.uniform(-0.5, 0.5, N) * ds_bg
    if nv == 3:
        sat = f_old == 0
        u_new[2, sat] = np.abs(u_new[2, sat] + rng.uniform(-0.5, 0.5, int(sat.sum())) * ds_bg)
        u_new[2, ~sat] *= rng.uniform(0.97, 1.03, int((~sat).sum()))
        # a few cells switch state, saturated -> undersaturated (only where
        # little gas was present) and back
        flip = rng.random(N) < 0.002
        to_un = flip & sat & (u_old[2] < 0.5 * ds_bg)
        to_sat = flip & ~sat
        f_new[to_un] = 1
        u_new[2, to_un] = 0.5 * float(np.max(g.tab_Rs))
        f_new[to_sat] = 0
        u_new[2, to_sat] = 0.0
    for (ci, cj, ck, radius, phase) in fronts:
        r = np.sqrt((i - ci) ** 2 + (j - cj) ** 2 + (k - ck) ** 2)
        on = np.abs(r - radius) < width
        if phase == 2 and nv == 3:
            on &= f_new == 0
            u_new[2, on] += ds_front
        else:
            u_new[1, on] += ds_front
    return State(u_new=u_new, flag_new=f_new, u_old=u_old, flag_old=f_old, dt=dt)


def addm_2d(seed=7, n=4000, radius_gas=None, radius_water=None):
    """The two-dimensional flood used for the adaptive coupling: an n x n x 1
    three-phase grid of 20 ft cells (n = 4000: 16 million cells), four
    injectors at (n/4, n/4), (n/4, 3n/4), (3n/4, n/4), (3n/4, 3n/4) and nine
    producers at the corners, edge midpoints and centre, ln k ~ N(ln 100, 1),
    phi ~ U(0.15, 0.3).  The state pair has a gas front (radius n/8) and a
    water front (radius n/16) around every injector."""
    rng = np.random.default_rng(seed)
    N = n * n
    lnk = rng.normal(math.log(100.0), 1.0, N)
    phi = rng.uniform(0.15, 0.3, N)
    g = make_grid(n, n, 1, lnk, phi, [], dx=20.0, dy=20.0, dz=20.0)
    q1, q3 = n // 4 - 1, (3 * n) // 4 - 1
    inj = [(q1, q1), (q1, q3), (q3, q1), (q3, q3)]
    edge = [0, n // 2 - 1, n - 1]
    g.wells = [Well(kind=1, phase=2, p_bh=5500.0, cells=g.column(a, b)) for (a, b) in inj]
    g.wells += [Well(kind=0, phase=0, p_bh=3500.0, cells=g.column(a, b)) for a in edge for b in edge]
    rg = n / 8.0 if radius_gas is None else radius_gas
    rw = n / 16.0 if radius_water is None else radius_water
    fronts = [(a, b, 0, rg, 2) for (a, b) in inj] + [(a, b, 0, rw, 0) for (a, b) in inj]
    return g, front_state(g, seed + 1, fronts)
