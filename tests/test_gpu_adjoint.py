"""Newton stepping and the multi-step adjoint on the GPU.

* one GPU Newton step (linearise, BiCGSTAB, update with chop and phase
  switch) reaches the state the oracle's Newton step (direct solve) reaches;
* the GPU solver meets its tolerance on the oracle's own Jacobian;
* the checkpointed multi-step gradient of the well-rate mismatch matches the
  oracle's dense adjoint on a small grid, and central differences of the GPU
  forward loss on the 100x100x10 history-matching case;
* the torch.autograd.Function returns that gradient.
"""
import copy

import numpy as np
import pytest

from _gpu_common import need_gpu, torch
from oracle.adjoint import loss_and_gradient, simulate
from oracle.linearize import linearize as oracle_linearize
from oracle.newton import newton_step as oracle_newton_step
from oracle.spmv import bsr_spmv
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def mods():
    need_gpu()
    from paper_2406_10862_gb300 import fim, ocp
    ocp.load()
    return ocp, fim


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_bicgstab_solves_the_oracle_jacobian():
    ocp, fim = mods()
    g, s = W.tiny(9, 8, 4, seed=120)
    o = oracle_linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt)
    grid = ocp.Grid(g)
    b = np.random.default_rng(0).normal(size=3 * g.N)
    rp, ci = o["row_ptr"], o["col_idx"]
    diag = [o["val"][rp[c] + list(ci[rp[c]:rp[c + 1]]).index(c)] for c in range(g.N)]
    for transpose in (False, True):
        x = torch.zeros(3 * g.N, dtype=torch.float64, device="cuda")
        st, it, rr = grid.bicgstab(T(o["val"].ravel()), T(b), x, 1e-12, 2000, transpose=transpose)
        res, _ = bsr_spmv(rp, ci, o["val"], x.cpu().numpy(), alpha=-1.0, beta=1.0, y=b, transpose=transpose)
        # the promised criterion: the residual scaled by the inverse diagonal blocks
        D = [d.T if transpose else d for d in diag]
        scaled = np.concatenate([np.linalg.solve(D[c], res[3 * c:3 * c + 3]) for c in range(g.N)])
        sb = np.concatenate([np.linalg.solve(D[c], b[3 * c:3 * c + 3]) for c in range(g.N)])
        assert np.linalg.norm(scaled) <= 1e-11 * np.linalg.norm(sb) and it > 0


@pytest.mark.parametrize("nphase,seed,dt", [(3, 121, 2.0), (2, 125, 1.0)])
def test_newton_step_reaches_the_oracle_state(nphase, seed, dt):
    ocp, fim = mods()
    g, s = W.tiny(6, 5, 3, nphase=nphase, seed=seed, frac_unsat=0.0)
    u_ref, f_ref, _, _ = oracle_newton_step(g, s.u_old, s.flag_old, dt)
    grid = ocp.Grid(g)
    st = fim.Stepper(grid)
    u, f = st.step(T(s.u_old.ravel()), T(s.flag_old), dt)
    u = u.cpu().numpy().reshape(nphase, g.N)
    assert np.array_equal(f.cpu().numpy(), f_ref)
    np.testing.assert_allclose(u[0], u_ref[0], rtol=0, atol=1e-6)
    np.testing.assert_allclose(u[1:], u_ref[1:], rtol=0, atol=1e-8 * max(1.0, np.abs(u_ref[1:]).max()))


def test_multistep_gradient_matches_the_oracle_adjoint():
    ocp, fim = mods()
    truth, s = W.tiny(5, 4, 3, seed=122, frac_unsat=0.0)
    prior = copy.deepcopy(truth)
    prior.lnk = truth.lnk + np.random.default_rng(123).normal(0.0, 0.3, truth.N)
    dt, nsteps = 2.0, 4
    states = simulate(truth, s.u_old, s.flag_old, dt, nsteps)
    q_obs = []
    for n in range(1, nsteps + 1):
        q_obs.append(oracle_linearize(truth, states[n][0], states[n][1], states[n - 1][0], states[n - 1][1],
                                      dt)["well_rate"])
    q_obs = np.array(q_obs)
    q_scale = np.abs(q_obs).max(axis=(0, 1)) + 1e-30
    loss_ref, g_ref, _ = loss_and_gradient(prior, s.u_old, s.flag_old, dt, nsteps, q_obs, q_scale)
    grid = ocp.Grid(prior)
    hm = fim.HistoryMatch(grid, T(s.u_old.ravel()), T(s.flag_old), dt, nsteps, q_obs=T(q_obs),
                          q_scale=T(q_scale), checkpoint=2)
    lnk = T(prior.lnk)
    loss, ckpts, _ = hm.run(lnk)
    assert sorted(ckpts) == [0, 2]
    assert float(loss) == pytest.approx(loss_ref, rel=1e-8)
    g_gpu = hm.gradient(lnk, ckpts).cpu().numpy()
    np.testing.assert_allclose(g_gpu, g_ref, rtol=1e-6, atol=1e-7 * np.abs(g_ref).max())
    # the same through autograd
    x = lnk.clone().requires_grad_(True)
    L = fim.HistoryMatchLoss.apply(x, hm)
    L.backward()
    np.testing.assert_allclose(x.grad.cpu().numpy(), g_gpu, rtol=1e-12, atol=1e-14 * np.abs(g_gpu).max())


def test_history_match_gradient_against_finite_differences():
    """The 100x100x10, 20-step case: adjoint gradient vs central differences
    (h = 1e-4 in ln k) of the GPU forward loss on 50 random cells and the six
    cells of largest gradient."""
    ocp, fim = mods()
    g, s, lnk_truth, lnk_prior, dt, nsteps = W.history_match()
    grid = ocp.Grid(g)
    u0, f0 = T(s.u_old.ravel()), T(s.flag_old)
    hm = fim.HistoryMatch(grid, u0, f0, dt, nsteps, checkpoint=5)
    _, _, rates = hm.run(T(lnk_truth))
    q_obs = torch.stack(rates)
    hm.q_obs = q_obs
    hm.q_scale = q_obs.abs().amax(dim=(0, 1)) + 1e-30
    lnk = T(lnk_prior)
    loss, ckpts, _ = hm.run(lnk)
    grad = hm.gradient(lnk, ckpts)
    gmax = float(grad.abs().max())
    cells = list(np.argsort(-np.abs(grad.cpu().numpy()))[:6]) + \
        list(np.random.default_rng(124).choice(g.N, 50, replace=False))
    h = 1e-4
    for c in cells:
        lp, lm = lnk.clone(), lnk.clone()
        lp[c] += h
        lm[c] -= h
        fd = (float(hm.run(lp)[0]) - float(hm.run(lm)[0])) / (2 * h)
        assert fd == pytest.approx(float(grad[c]), rel=1e-4, abs=1e-5 * gmax), (c, fd, float(grad[c]))
