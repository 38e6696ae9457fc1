"""Newton time stepping and the multi-step adjoint on top of the C library.

The FIM nonlinear iteration of Sec. 3.2.5 -- linearise (``ocp_linearize``),
solve (``ocp_bicgstab``), update with chop and phase switch
(``ocp_newton_update``), test convergence -- repeated over time steps, and the
reverse pass of a loss on the well rates.  ``Stepper.step_wells`` runs the
same iteration with the wells' bottom-hole pressures as unknowns under
pressure or rate control (``ocp_linearize_wells``, ``ocp_bicgstab_wells``,
``ocp_well_update``) and a residual-norm convergence test
(``ocp_residual_norms``); ``Stepper.step_pn`` runs it in the paper's own
unknowns, pressure and component amounts with the volume balance
(``ocp_linearize_pn``, ``ocp_pn_update``, ``ocp_pn_norms``); ``impec_step``
is one IMPEC step in the same unknowns.  The gradient with respect to the
log-permeability field is

    dL/d ln k = sum_n [ dl_n/d ln k - lambda_n^T dR_n/d ln k ],
    J_n^T lambda_n = dl_n/du_n - (dR_{n+1}/du_n)^T lambda_{n+1},

with every product by a Jacobian done by the library's kernels
(``ocp_adjoint_vjp``, ``ocp_well_rates_vjp``, transposed ``ocp_bicgstab``).
States are kept only at checkpoints (every ``checkpoint`` steps) and the
steps in between are recomputed during the reverse pass; the kernels are
deterministic, so the recomputed states are bit-identical to the forward
ones.  ``HistoryMatchLoss`` wraps it as a ``torch.autograd.Function``.

The vector bookkeeping between library calls (sums of cotangents, the
layout change from variable-major to block-interleaved) uses torch tensor
operations on the device; all Jacobian work runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses

import torch

from . import ocp


class NewtonFailure(RuntimeError):
    pass


@dataclasses.dataclass
class NewtonOptions:
    rtol: float = 1e-12          # linear solve, relative
    maxit: int = 1000            # linear iterations
    tol_p: float = 1e-7          # psi (and scf/stb for R_s)
    tol_s: float = 1e-10         # saturation
    max_newton: int = 30
    ds_max: float = 0.2
    tol_cnv: float = 1e-9        # scaled residual, per pore volume (with well unknowns)
    tol_well: float = 1e-9       # well residual, relative to the rate target (psi under pressure control)
    tol_vol: float = 1e-12       # volume-balance residual, (P, N) unknowns


class Stepper:
    """Backward-Euler Newton steps on one grid."""

    def __init__(self, grid: ocp.Grid, opts: NewtonOptions | None = None):
        self.g = grid
        self.o = opts or NewtonOptions()
        nb, N = grid.nb, grid.N
        self.r = grid.empty(nb * N)
        self.val = grid.empty(grid.nnzb * nb * nb)
        self.ff = grid.empty(3 * nb * N)
        self.du = grid.empty(nb * N)
        self.work = grid.solver_work()
        self.dmax = grid.empty(4)
        self.nsw = torch.zeros(1, dtype=torch.int32, device=grid.device)
        self.newton_iters = 0
        self.linear_iters = 0

    def step(self, u_old, f_old, dt):
        """Solve R(u; u_old) = 0; returns (u, flag)."""
        g, o = self.g, self.o
        u, f = u_old.clone(), f_old.clone()
        for it in range(1, o.max_newton + 1):
            g.linearize(u, f, u_old, f_old, dt, self.r, self.val, self.ff)
            self.du.zero_()
            _, li, _ = g.bicgstab(self.val, self.r, self.du, o.rtol, o.maxit, work=self.work)
            self.linear_iters += li
            g.newton_update(u, f, self.du, -1.0, o.ds_max, self.dmax, self.nsw)
            d = self.dmax.cpu().tolist()
            nsw = int(self.nsw.item())
            self.newton_iters += 1
            # du_max holds nb + 1 maxima: p, S_w, then S_g and R_s with three phases
            small = d[0] < o.tol_p and d[1] < o.tol_s and (g.nb == 2 or (d[2] < o.tol_s and d[3] < o.tol_p))
            if nsw == 0 and small:
                st = g.status()
                if st != 0:
                    raise NewtonFailure("device status %d" % st)
                return u, f
        raise NewtonFailure("Newton did not converge in %d iterations" % o.max_newton)

    def step_wells(self, u_old, f_old, dt, p_bh, ctrl):
        """One step with the bottom-hole pressures as unknowns (``ctrl`` is a
        device ocp_well_ctrl array, see ``ocp.well_controls``; a well that
        reaches its pressure limit is switched to pressure control in it).
        Converged when the scaled residuals (``ocp_residual_norms``) are below
        tol_cnv / tol_well at an iterate whose update switched nothing.
        Returns (u, flag, p_bh, linearisations)."""
        g, o = self.g, self.o
        nb, nw = g.nb, g.nwell
        u, f, p = u_old.clone(), f_old.clone(), p_bh.clone()
        if not hasattr(self, "_wb"):
            self._wb = {"residual": self.r, "bsr_val": self.val, "well_res": g.empty(max(nw, 1)),
                        "well_b": g.empty(max(g.nperf, 1) * nb), "well_c": g.empty(max(g.nperf, 1) * nb),
                        "well_d": g.empty(max(nw, 1))}
            self._dp = g.empty(max(nw, 1))
            self._norms = g.empty(4)
            self._dpmax = g.empty(1)
            self._nsw_w = torch.zeros(1, dtype=torch.int32, device=g.device)
        wb = self._wb
        nsw = 1
        for it in range(1, o.max_newton + 1):
            g.linearize_wells(u, f, u_old, f_old, dt, p, ctrl, out=wb)
            nrm = g.residual_norms(wb["residual"], dt, wb["well_res"], ctrl, self._norms).cpu().tolist()
            if nsw == 0 and max(nrm[:nb]) < o.tol_cnv and nrm[3] < o.tol_well:
                st = g.status()
                if st != 0:
                    raise NewtonFailure("device status %d" % st)
                return u, f, p, it
            self.du.zero_()
            self._dp.zero_()
            _, li, _ = g.bicgstab_wells(wb["bsr_val"], wb["well_b"], wb["well_c"], wb["well_d"], wb["residual"],
                                        wb["well_res"], self.du, self._dp, o.rtol, o.maxit, work=self.work)
            self.linear_iters += li
            g.newton_update(u, f, self.du, -1.0, o.ds_max, self.dmax, self.nsw)
            g.well_update(p, self._dp, -1.0, ctrl, self._dpmax, self._nsw_w)
            self.newton_iters += 1
            nsw = int(self.nsw.item()) + int(self._nsw_w.item())
        raise NewtonFailure("Newton did not converge in %d iterations" % o.max_newton)

    def step_pn(self, pn_old, dt, pn_start=None):
        """One step in the (P, N) unknowns (Sec. 2.1): linearise and eliminate
        the volume rows (``ocp_linearize_pn``), solve the reduced system,
        recover N_w and update (``ocp_pn_update``).  Converged when the scaled
        component residuals are below tol_cnv and the volume residuals below
        tol_vol (``ocp_pn_norms``).  Returns (pn, flag, linearisations)."""
        g, o = self.g, self.o
        nb, N = g.nb, g.N
        pn = (pn_old if pn_start is None else pn_start).clone()
        if not hasattr(self, "_pnb"):
            self._pnb = {"residual": self.r, "bsr_val": self.val, "residual_full": g.empty((nb + 1) * N)}
            self._pn_norms = g.empty(4)
            self._pn_dmax = g.empty(nb + 1)
        for it in range(1, o.max_newton + 1):
            b = self._pnb = g.linearize_pn(pn, pn_old, dt, out=self._pnb)
            nrm = g.pn_norms(b["residual_full"], dt, self._pn_norms).cpu().tolist()
            if max(nrm[:nb]) < o.tol_cnv and nrm[3] < o.tol_vol:
                st = g.status()
                if st != 0:
                    raise NewtonFailure("device status %d" % st)
                return pn, b["flag"].clone(), it
            self.du.zero_()
            _, li, _ = g.bicgstab(b["bsr_val"], b["residual"], self.du, o.rtol, o.maxit, work=self.work)
            self.linear_iters += li
            g.pn_update(pn, self.du, -1.0, b["elim"], self._pn_dmax)
            self.newton_iters += 1
        raise NewtonFailure("Newton did not converge in %d iterations" % o.max_newton)

    def linearize_at(self, u, f, u_old, f_old, dt):
        self.g.linearize(u, f, u_old, f_old, dt, self.r, self.val, self.ff)
        return self.r, self.val, self.ff


def impec_step(grid, pn_old, dt, rtol=1e-13, maxit=2000, work=None):
    """One IMPEC step in the (P, N) unknowns: the pressure system
    (``ocp_impec_pressure``), its Jacobi-preconditioned BiCGSTAB solve
    (``ocp_bicgstab_scalar``) and the explicit update (``ocp_impec_update``).
    Returns (pn_new, dP, linear iterations)."""
    val, rhs = grid.impec_pressure(pn_old, dt)
    dp = torch.zeros(grid.N, dtype=torch.float64, device=grid.device)
    _, it, _ = grid.bicgstab_scalar(val, rhs, dp, rtol, maxit, work=work)
    return grid.impec_update(pn_old, dp, dt), dp, it


def to_blocks(v, nb, N):
    """Variable-major [nb*N] -> block-interleaved [nb*N]."""
    return v.view(nb, N).t().contiguous().view(-1)


class HistoryMatch:
    """Squared well-rate mismatch over a fixed sequence of steps,
    L = sum_n sum_w sum_e ((q_we(u_n) - q_obs_nwe) / q_scale_e)^2."""

    def __init__(self, grid, u0, f0, dt, nsteps, q_obs=None, q_scale=None, checkpoint=5, opts=None):
        self.g = grid
        self.u0, self.f0 = u0, f0
        self.dt, self.T = dt, nsteps
        self.q_obs, self.q_scale = q_obs, q_scale
        self.ck = checkpoint
        self.stepper = Stepper(grid, opts)

    def rates(self, u, f):
        return self.g.well_rates(u, f).view(self.g.nwell, self.g.nb).clone()

    def run(self, lnk, record=False):
        """Forward pass: returns (loss, checkpoints, rates per step)."""
        self.g.update_perm(lnk)
        u, f = self.u0.clone(), self.f0.clone()
        ckpts = {0: (u.clone(), f.clone())}
        rates, loss = [], torch.zeros((), dtype=torch.float64, device=self.g.device)
        for n in range(1, self.T + 1):
            u, f = self.stepper.step(u, f, self.dt)
            q = self.rates(u, f)
            rates.append(q)
            if self.q_obs is not None:
                loss = loss + (((q - self.q_obs[n - 1]) / self.q_scale) ** 2).sum()
            if n % self.ck == 0 and n < self.T:
                ckpts[n] = (u.clone(), f.clone())
        return loss, ckpts, rates

    def gradient(self, lnk, ckpts):
        """Reverse pass: dL/d ln k from the checkpoints of ``run(lnk)``."""
        g, nb, N = self.g, self.g.nb, self.g.N
        g.update_perm(lnk)
        st = self.stepper
        g_lnk = torch.zeros(N, dtype=torch.float64, device=g.device)
        carry = None                        # (dR_{n+1}/du_n)^T lambda_{n+1}, variable-major
        starts = sorted(ckpts)
        for s0 in reversed(starts):
            s1 = min(s0 + self.ck, self.T)
            states = [ckpts[s0]]
            for n in range(s0 + 1, s1 + 1):  # recompute the segment
                states.append(st.step(states[-1][0], states[-1][1], self.dt))
            for n in range(s1, s0, -1):
                u, f = states[n - s0]
                up, fp = states[n - s0 - 1]
                _, val, ff = st.linearize_at(u, f, up, fp, self.dt)
                q = self.rates(u, f)
                qbar = (2.0 * (q - self.q_obs[n - 1]) / self.q_scale ** 2).contiguous().view(-1)
                rhs = torch.zeros(nb * N, dtype=torch.float64, device=g.device)
                g.well_rates_vjp(u, f, qbar, g_u=rhs, g_lnk=g_lnk)
                if carry is not None:
                    rhs -= carry
                rhs_b = to_blocks(rhs, nb, N)
                lam = torch.zeros_like(rhs_b)
                g.bicgstab(val, rhs_b, lam, st.o.rtol, st.o.maxit, transpose=True, work=st.work)
                out = g.adjoint_vjp(u, f, up, fp, self.dt, val, ff, lam, want=("uold", "lnk"))
                g_lnk -= out["lnk"]
                carry = out["uold"]
        return g_lnk


class HistoryMatchLoss(torch.autograd.Function):
    """loss = HistoryMatchLoss.apply(lnk, history_match); differentiable in lnk."""

    @staticmethod
    def forward(ctx, lnk, hm):
        loss, ckpts, _ = hm.run(lnk.detach())
        ctx.hm = hm
        ctx.ckpts = ckpts
        ctx.save_for_backward(lnk)
        return loss

    @staticmethod
    def backward(ctx, gout):
        (lnk,) = ctx.saved_tensors
        return ctx.hm.gradient(lnk.detach(), ctx.ckpts) * gout, None
