"""Multi-step adjoint of a well-rate mismatch, in dense linear algebra (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

For states u_n defined by R_n(u_n; u_{n-1}, ln k) = 0 (one FIM step each,
``oracle.newton.newton_step``) and L = sum_n l_n(u_n, ln k) with
l_n = sum_w sum_e ((q_we(u_n) - q_obs)/q_scale_e)^2, the gradient is
dL/d ln k = sum_n [dl_n/d ln k - lambda_n^T dR_n/d ln k] with
J_n^T lambda_n = dl_n/du_n - (dR_{n+1}/du_n)^T lambda_{n+1}.  Every matrix
here is formed densely from the oracle's dual-number derivatives and every
solve is numpy's dense LU, so this is only for tiny grids.
"""
from __future__ import annotations

import numpy as np

from .linearize import linearize
from .newton import newton_step
from .spmv import bsr_to_dense


def simulate(spec, u0, f0, dt, nsteps):
    states = [(np.array(u0, dtype=np.float64), np.array(f0).copy())]
    for _ in range(nsteps):
        u, f, _, _ = newton_step(spec, states[-1][0], states[-1][1], dt)
        states.append((u, f))
    return states


def loss_and_gradient(spec, u0, f0, dt, nsteps, q_obs, q_scale):
    nv = nb = int(spec.nphase)
    N = int(spec.nx * spec.ny * spec.nz)
    L = 2 * nv + 2
    states = simulate(spec, u0, f0, dt, nsteps)
    loss = 0.0
    g_lnk = np.zeros(N)
    carry = np.zeros(N * nb)                  # (dR_{n+1}/du_n)^T lambda_{n+1}, block-interleaved
    for n in range(nsteps, 0, -1):
        u, f = states[n]
        up, fp = states[n - 1]
        o = linearize(spec, u, f, up, fp, dt, mode="all", lam=np.zeros((N, nb)))
        q = o["well_rate"]
        loss += float((((q - q_obs[n - 1]) / q_scale) ** 2).sum())
        qbar = 2.0 * (q - q_obs[n - 1]) / q_scale ** 2
        dl_du = np.zeros((N, nb))
        for w, (cells, gq) in enumerate(o["well_grad"]):
            for e in range(nb):
                np.add.at(dl_du, cells, qbar[w, e] * gq[:, e, :nv])
                np.add.at(g_lnk, cells, qbar[w, e] * gq[:, e, 2 * nv])
        J = bsr_to_dense(o["row_ptr"], o["col_idx"], o["val"])
        lam = np.linalg.solve(J.T, dl_du.ravel() - carry)
        ov = linearize(spec, u, f, up, fp, dt, mode="all", lam=lam.reshape(N, nb))
        g_lnk -= ov["g_lnk"]
        carry = ov["g_uold"].T.ravel()
    return loss, g_lnk, states
