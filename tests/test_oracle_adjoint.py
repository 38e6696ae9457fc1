"""Pin of the oracle's multi-step adjoint: its gradient of the well-rate
mismatch with respect to ln k equals central differences of the loss computed
by forward simulation alone (Newton steps, no derivatives of the adjoint)."""
import copy

import numpy as np
import pytest

from oracle.adjoint import loss_and_gradient, simulate
from oracle.linearize import linearize
from paper_2406_10862_gb300 import workloads as W


def observed(spec, u0, f0, dt, nsteps):
    states = simulate(spec, u0, f0, dt, nsteps)
    q = []
    for n in range(1, nsteps + 1):
        o = linearize(spec, states[n][0], states[n][1], states[n - 1][0], states[n - 1][1], dt)
        q.append(o["well_rate"])
    return np.array(q)


@pytest.mark.slow
@pytest.mark.parametrize("nphase", [3, 2])
def test_multistep_adjoint_matches_finite_differences(nphase):
    truth, s = W.tiny(3, 3, 2, nphase=nphase, seed=31, frac_unsat=0.0)
    prior = copy.deepcopy(truth)
    prior.lnk = truth.lnk + np.random.default_rng(32).normal(0.0, 0.3, truth.N)
    u0, f0, dt, T = s.u_old, s.flag_old, 2.0, 3
    q_obs = observed(truth, u0, f0, dt, T)
    q_scale = np.abs(q_obs).max(axis=(0, 1)) + 1e-30
    loss, g, _ = loss_and_gradient(prior, u0, f0, dt, T, q_obs, q_scale)
    assert loss > 0
    h = 1e-5
    for c in (0, 4, 8, 13, prior.N - 1):
        lp, lm = copy.deepcopy(prior), copy.deepcopy(prior)
        lp.lnk[c] += h
        lm.lnk[c] -= h
        fd = (loss_and_gradient(lp, u0, f0, dt, T, q_obs, q_scale)[0] -
              loss_and_gradient(lm, u0, f0, dt, T, q_obs, q_scale)[0]) / (2 * h)
        assert fd == pytest.approx(g[c], rel=2e-5, abs=2e-6 * np.abs(g).max())
