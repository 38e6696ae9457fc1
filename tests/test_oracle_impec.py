"""Pins of the IMPEC oracle (pressure from the linearised volume balance, then
an explicit conservative update of the amounts): conservation, a state at
rest stays at rest, the pressure equation is affine with the matrix the
oracle returns, the step agrees with the fully implicit step to second order
in dt, the volume balance after the step is off only to second order, and
planted mistakes are caught."""
import importlib
import importlib.util
import os
import shutil
import sys

import numpy as np
import pytest

from paper_2406_10862_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load(tmp_path=None, mutation=None, tag="base"):
    if mutation is None:
        import oracle.impec as im
        import oracle.pn as pn
        return im, pn
    dst = tmp_path / ("oracle_im_" + tag)
    shutil.copytree(os.path.join(ROOT, "oracle"), dst)
    f = dst / "impec.py"
    src = f.read_text()
    old, new = mutation
    assert src.count(old) == 1, old
    f.write_text(src.replace(old, new))
    name = "oracle_im_mut_" + tag
    spec = importlib.util.spec_from_file_location(name, dst / "__init__.py", submodule_search_locations=[str(dst)])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    return importlib.import_module(name + ".impec"), importlib.import_module(name + ".pn")


def _state(nphase=3, wells=True, seed=4, nz=3):
    g, s = W.tiny(6, 5, nz, nphase=nphase, seed=seed, frac_unsat=0.3 if nphase == 3 else 0.0, rs_hi=0.7,
                  wells=wells)
    return g, s


def pin_conservation(im, pn):
    for nphase in (2, 3):
        g, s = _state(nphase)
        x0 = pn.natural_to_pn(g, s.u_new, s.flag_new)
        dt = 0.3
        x1, dP, A, E0 = im.impec_step(g, x0, dt)
        old = im._old_level(g, x0)
        flux, src = im._fluxes_and_sources(g, x0, old, pn.D.const(dP, g.N, 1))
        vdt = g.dx * g.dy * g.dz / 5.614583 / dt
        for e in range(nphase):
            lhs = ((x1[1 + e] - x0[1 + e]) * vdt).sum()
            rhs = src[e].v.sum()
            scale = np.abs(src[e].v).sum() + np.abs(flux[e].v).sum() + 1e-300
            assert abs(lhs - rhs) <= 1e-11 * scale
            # and the faces cancel: the summed net outflow is zero
            assert abs(flux[e].v.sum()) <= 1e-12 * (np.abs(flux[e].v).sum() + 1e-300)


def pin_rest_stays_at_rest(im, pn):
    # one layer (no gravity head), a uniform consistent state, no wells
    g, s = _state(3, wells=False, nz=1)
    u = s.u_old.copy()
    x0 = pn.natural_to_pn(g, u, s.flag_old)
    x1, dP, A, E0 = im.impec_step(g, x0, 1.0)
    assert np.all(np.abs(dP) <= 1e-9)          # psi; eq. 4 is met to rounding only
    assert np.allclose(x1[1:], x0[1:], rtol=1e-14, atol=1e-16)


def pin_pressure_equation_is_affine_with_its_matrix(im, pn):
    g, s = _state(3)
    x0 = pn.natural_to_pn(g, s.u_new, s.flag_new)
    dt = 0.5
    A, E0, _, _, old = im.pressure_system(g, x0, dt)
    rng = np.random.default_rng(7)
    d = rng.normal(0.0, 5.0, g.N)
    flux, src = im._fluxes_and_sources(g, x0, old, pn.D.const(d, g.N, 1))
    vdt = g.dx * g.dy * g.dz / 5.614583 / dt
    E = (old["phi"] - old["V_f"]) * vdt + d * (old["phi_P"] - old["V_f_P"]) * vdt
    for e in range(3):
        E = E + (flux[e].v - src[e].v) * old["w"][:, e]
    ref = E0 + A @ d
    assert np.allclose(E, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    # the 7-point pattern: no entry outside a cell's faces
    assert A.nnz <= 7 * g.N


def pin_second_order_agreement_with_the_implicit_step(im, pn):
    g, s = _state(3, wells=False)
    x0 = pn.natural_to_pn(g, s.u_new, s.flag_new)
    errs = []
    for dt in (1e-3, 1e-4):
        x1, _, _, _ = im.impec_step(g, x0, dt)
        xf, _, _ = pn.newton_step_pn(g, x0, dt)
        errs.append(np.abs(x1[0] - xf[0]).max())
    ratio = errs[0] / errs[1]
    assert 60.0 < ratio < 160.0, ratio


def pin_volume_balance_error_is_second_order(im, pn):
    # all-saturated state, steps small enough to stay clear of table and
    # relative-permeability kinks
    g, s = W.tiny(6, 5, 3, nphase=3, seed=4, frac_unsat=0.0, wells=False)
    x0 = pn.natural_to_pn(g, s.u_new, s.flag_new)
    errs = []
    for dt in (1e-3, 1e-4):
        x1, _, _, _ = im.impec_step(g, x0, dt)
        o = pn.linearize_pn(g, x1, x0, dt)
        errs.append(np.abs(o["R"][:, 3]).max())
    assert errs[0] / errs[1] > 30.0, errs


PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__[4:])
def test_pin(pin):
    im, pn = _load()
    pin(im, pn)


MUTATIONS = [
    ("E = E + (flux[e] - src[e]) * old[\"w\"][:, e]", "E = E + (flux[e] + src[e]) * old[\"w\"][:, e]"),
    ("dP * ((old[\"phi_P\"] - old[\"V_f_P\"]) * vdt)", "dP * ((old[\"phi_P\"] + old[\"V_f_P\"]) * vdt)"),
    ("up_i = dphi_old >= 0.0", "up_i = dphi_old < 0.0"),
    ("dphi = (Pi - Pj) + (off_i - off_j - gamma * dz_ij)", "dphi = (Pi - Pj) + (off_i - off_j + gamma * dz_ij)"),
    ("pn_new[1 + e] = pn_old[1 + e] + (src[e].v - flux[e].v) / vdt",
     "pn_new[1 + e] = pn_old[1 + e] + (src[e].v - flux[e].v) * vdt"),
    ("comp.append(F[\"g\"] + F[\"o\"] * rs_up)", "comp.append(F[\"g\"])"),
]


@pytest.mark.filterwarnings("ignore::scipy.sparse.linalg.MatrixRankWarning")
@pytest.mark.parametrize("k", range(len(MUTATIONS)))
def test_planted_mistake_is_caught(tmp_path, k):
    im, pn = _load(tmp_path, MUTATIONS[k], "m%d" % k)
    failed = []
    for pin in PINS:
        try:
            with np.errstate(all="ignore"):
                pin(im, pn)
        except (AssertionError, RuntimeError, ValueError, FloatingPointError, np.linalg.LinAlgError, IndexError,
                ZeroDivisionError):
            failed.append(pin.__name__)
    assert failed, "mutation %r passed every pin" % (MUTATIONS[k][0],)
