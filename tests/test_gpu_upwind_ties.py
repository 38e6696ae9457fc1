"""GPU parity at upwind ties: hydrostatic states, where a phase's potential
difference across every vertical face is zero to within rounding.

There the sign of the potential difference, and with it the upwind cell that
the rule "upwind = i where the potential difference is >= 0" picks (Darcy's
law, eq. 2, in two-point form), is decided by rounding alone: the library and
the oracle evaluate the difference in different orders and may land on
opposite sides of zero.  Both results are correct -- the flux vanishes either
way and each side's one-sided derivative is exact -- but the Jacobian blocks
of the two choices differ by T (lambda_i - lambda_j), far beyond the parity
tolerance.  So these tests compare what is unique and check that the rest is
valid: for every tied face the library's off-diagonal block tells which side
it took; the oracle is then evaluated with exactly those choices, allowed
only on faces whose potential difference is within a few units of rounding
of zero (its magnitude scale), and everything is compared at the usual
1e-12 / 1e-10 tolerances.  Faces that are not tied must match the oracle's
own choice.
"""
import numpy as np
import pytest

from _gpu_common import RTOL_J, RTOL_R, assert_scaled_close, gpu_linearize, need_gpu
from oracle import blackoil as bo
from oracle.dual import D
from oracle.linearize import bsr_pattern, face_pairs, linearize as oracle_linearize
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
TIE_ULPS = 16.0          # |dphi| <= TIE_ULPS * eps * magnitude scale counts as a tie


def equilibrium_state(g, phase, sw=0.3, x=0.05, flag=0, seed=0):
    """A state at rest for one phase: saturations uniform, the top layer's
    pressure drawn per column, and every deeper layer's pressure solved (to
    a fixed point in FP64) so that the phase's potential difference across
    each vertical face, with the mean of the two cells' densities, is zero.
    The densities are the oracle's; lateral pressure differences keep the
    horizontal faces untied."""
    rng = np.random.default_rng(seed)
    ncol = g.nx * g.ny
    p = np.zeros((g.nz, ncol))
    p[0] = 4000.0 + rng.uniform(0.0, 800.0, ncol)
    key = "rho_" + phase

    def rho(pp):
        n = len(pp)
        pr = bo.cell_properties(g, D.seed(pp, 1, 0), D.const(sw, n, 1), D.const(x, n, 1),
                                np.full(n, flag, dtype=np.int8), np.full(n, 0.2))
        return pr[key].v

    for k in range(g.nz - 1):
        r0 = rho(p[k])
        nxt = p[k] + r0 * bo.GRAV * g.dz
        for _ in range(100):
            new = p[k] + (r0 + rho(nxt)) * (0.5 * bo.GRAV) * g.dz
            if np.array_equal(new, nxt):
                break
            nxt = new
        p[k + 1] = nxt
    u = np.zeros((3, g.N))
    u[0], u[1], u[2] = p.ravel(), sw, x
    f = np.full(g.N, flag, dtype=np.int8)
    return W.State(u_new=u, flag_new=f, u_old=u.copy(), flag_old=f.copy(), dt=1.0)


def check_with_ties(g, s, phases):
    from paper_2406_10862_gb300 import ocp as O
    O.load()
    grid = O.Grid(g)
    r, v, ff, st = gpu_linearize(grid, s)
    assert st == 0
    nb = g.nphase
    v = v.reshape(-1, nb, nb)
    o = oracle_linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt)
    row_ptr, _, slot = bsr_pattern(g)
    tied = {}
    for d in range(3):
        for a in phases:
            dphi, mag = o["face_dphi"][(d, a)], o["face_dphi_mag"][(d, a)]
            tied[(d, a)] = np.abs(dphi) <= TIE_ULPS * EPS * mag
    # each tied face: which side did the library take?  Flip every tied face
    # in the oracle and keep, face by face, the branch closer to the library's
    # off-diagonal block (row i, column j), which only that face forms.
    o_flip = oracle_linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt, up_flip=tied)
    choice = {}
    n_tied = n_flipped = 0
    for (d, a), t in tied.items():
        fi, _ = face_pairs(g, d)
        blk = row_ptr[fi] + slot[4 + d][fi]

        def err(ref):
            e = np.abs(v[blk] - ref["val"][blk]) / (ref["val_mag"][blk] + 1e-300)
            return e.reshape(len(blk), -1).max(axis=1)

        flip = t & (err(o_flip) < err(o))
        choice[(d, a)] = flip
        n_tied += int(t.sum())
        n_flipped += int(flip.sum())
    o_sel = oracle_linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt, up_flip=choice)
    assert_scaled_close(r, o_sel["R"], o_sel["R_mag"], RTOL_R, "residual")
    assert_scaled_close(v, o_sel["val"], o_sel["val_mag"], RTOL_J, "jacobian")
    assert_scaled_close(ff, o_sel["face_flux"], o_sel["face_flux_mag"], RTOL_R, "face flux")
    return n_tied, n_flipped


@pytest.mark.parametrize("phase,flag", [("w", 0), ("o", 0), ("g", 0), ("o", 1)])
def test_equilibrium_of_one_phase(phase, flag):
    """Pressure at rest for water, oil (saturated and undersaturated) or gas
    on a 4x3x12 box with the synthetic, compressible fluid: every vertical
    face of that phase is a tie, and the phase's mobility differs between
    the layers, so the side taken matters to the Jacobian."""
    need_gpu()
    g, _ = W.tiny(4, 3, 12, seed=5, wells=False)
    x = 0.6 * float(np.max(g.tab_Rs)) * 0.5 if flag == 1 else 0.05
    s = equilibrium_state(g, phase, x=x, flag=flag, seed=7)
    n_tied, n_flipped = check_with_ties(g, s, ["w", "o", "g"])
    print("%s (flag %d): %d tied faces, %d taken on the other side by the library" % (phase, flag, n_tied,
                                                                                  n_flipped))
    assert n_tied >= (g.nz - 1) * g.nx * g.ny


def test_hydrostatic_incompressible_state():
    """The hydrostatic state of pin P3 on a multi-layer grid (flat tables,
    uniform saturations, water pressure p_0 + rho_w g z, wells off): every
    vertical water face is a tie; the residual is pure accumulation (zero)."""
    need_gpu()
    n = 20
    # flat oil and gas tables (the library requires an increasing R_s column,
    # which only moves the oil density; the tied phase is water)
    flat = dict(tab_Bo=np.full(n, 1.25), tab_Bg=np.full(n, 0.001), tab_muo=np.full(n, 0.8),
                tab_mug=np.full(n, 0.02), cw=0.0, cr=0.0, co_under=0.0, pcow_max=0.0, pcgo_max=0.0)
    g, _ = W.tiny(5, 4, 9, seed=23, wells=False, **flat)
    z = g.top_depth + (np.arange(g.N) // (g.nx * g.ny) + 0.5) * g.dz
    u = np.zeros((3, g.N))
    u[0] = 3000.0 + g.rho_wsc * g.bw_ref * bo.GRAV * z
    u[1] = 0.5
    u[2] = 0.1
    f = np.zeros(g.N, dtype=np.int8)
    s = W.State(u_new=u, flag_new=f, u_old=u.copy(), flag_old=f.copy(), dt=1.0)
    n_tied, n_flipped = check_with_ties(g, s, ["w", "o", "g"])
    print("hydrostatic water: %d tied faces, %d taken on the other side by the library" % (n_tied, n_flipped))
    assert n_tied >= (g.nz - 1) * g.nx * g.ny
