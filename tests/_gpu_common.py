"""Shared helpers of the GPU parity tests: moving seeded inputs to the device,
running the library and the oracle on the same inputs, and the tolerances.

Tolerances (FP64, differing summation order): every residual entry within
1e-12 and every Jacobian entry within 1e-10 of the oracle, relative to the
entry's magnitude scale -- the sum of the absolute values of the terms that
form it, carried through the oracle's dual numbers (``oracle.dual``).  The
scale is what bounds rounding differences between two evaluation orders of
the same sums; the plain relative error is meaningless where terms cancel.
"""
import numpy as np
import pytest

from paper_2406_10862_gb300 import workloads as W

torch = pytest.importorskip("torch")

RTOL_R = 1e-12
RTOL_J = 1e-10
RTOL_SPMV = 1e-13
RTOL_VJP = 1e-10


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev_state(s, device="cuda"):
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=device)
    return (f(s.u_new.ravel()), f(s.flag_new.astype(np.int8)), f(s.u_old.ravel()),
            f(s.flag_old.astype(np.int8)))


def gpu_linearize(grid, s, want_face_flux=True):
    un, fn, uo, fo = dev_state(s)
    r, v, ff = grid.linearize(un, fn, uo, fo, s.dt, want_face_flux=want_face_flux)
    st = grid.status()
    return r.cpu().numpy(), v.cpu().numpy(), (ff.cpu().numpy() if ff is not None else None), st


def assert_scaled_close(got, ref, mag, rtol, what):
    got = np.asarray(got).ravel()
    ref = np.asarray(ref).ravel()
    mag = np.asarray(mag).ravel()
    err = np.abs(got - ref)
    lim = rtol * mag + 1e-300
    bad = np.nonzero(err > lim)[0]
    if len(bad):
        k = bad[np.argmax(err[bad] / lim[bad])]
        raise AssertionError("%s: %d of %d entries off; worst index %d got %.17g ref %.17g scale %.3g "
                             "(err/scale %.3g)" % (what, len(bad), len(err), k, got[k], ref[k], mag[k],
                                                    err[k] / max(mag[k], 1e-300)))


def window(g, s, c, with_well_index=False):
    """The 3x3x3 (clipped) window around cell c as a grid of its own: the
    centre cell's residual row depends on nothing outside it.  With
    ``with_well_index`` also the original index of every well kept."""
    nx, ny, nz = g.nx, g.ny, g.nz
    i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
    i0, i1, j0, j1, k0, k1 = max(i - 1, 0), min(i + 2, nx), max(j - 1, 0), min(j + 2, ny), max(k - 1, 0), min(k + 2, nz)
    kk, jj, ii = np.meshgrid(np.arange(k0, k1), np.arange(j0, j1), np.arange(i0, i1), indexing="ij")
    cells = (ii + nx * (jj + ny * kk)).ravel()
    local = {int(x): n for n, x in enumerate(cells)}
    wells = []
    kept = []
    for iw, w in enumerate(g.wells):
        inside = [local[int(x)] for x in w.cells if int(x) in local]
        if inside:
            wells.append(W.Well(kind=w.kind, phase=w.phase, p_bh=w.p_bh, rw=w.rw, skin=w.skin,
                                cells=np.array(inside, dtype=np.int64)))
            kept.append(iw)
    h = W.GridDesc(**{f: getattr(g, f) for f in g.__dataclass_fields__})
    h.nx, h.ny, h.nz = i1 - i0, j1 - j0, k1 - k0
    h.top_depth = g.top_depth + k0 * g.dz
    h.lnk, h.phi, h.wells = g.lnk[cells], g.phi[cells], wells
    st = W.State(u_new=s.u_new[:, cells], flag_new=s.flag_new[cells], u_old=s.u_old[:, cells],
                 flag_old=s.flag_old[cells], dt=s.dt)
    centre = local[int(c)]
    if with_well_index:
        return h, st, centre, cells, kept
    return h, st, centre
