"""Slab partition of one grid over ranks, with ghost layers (Sec. 3.4).

Each rank owns a contiguous range of layers k0 <= k < k1 and builds a
sub-grid that adds one ghost layer on each side that has a neighbour rank.
Only the primary variables of the ghost layers are exchanged (point-to-point,
``torch.distributed`` send/recv: NCCL between GPUs, gloo on the CPU); the
ghost cells' properties are then recomputed locally by the linearisation, as
the paper describes for its ghost cells.  The rows of the owned cells in the
sub-grid's Jacobian have exactly the blocks, in the same order, as the same
rows of the whole grid's Jacobian, and every row sums its terms in a fixed
order, so the partitioned linearisation is bit-identical to the unpartitioned
one.  Well perforations are kept on the rank that owns their cell.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch
import torch.distributed as dist

from . import workloads as W


@dataclasses.dataclass
class Slab:
    rank: int
    world: int
    k0: int            # first owned layer
    k1: int            # one past the last owned layer
    lo: int            # ghost layers below k0 (0 or 1)
    hi: int            # ghost layers above k1 (0 or 1)
    nxy: int

    @property
    def owned(self):
        """Slice of the owned cells in the sub-grid's natural order."""
        return slice(self.lo * self.nxy, (self.lo + self.k1 - self.k0) * self.nxy)

    @property
    def global_cells(self):
        """Global natural index of every sub-grid cell."""
        return np.arange((self.k0 - self.lo) * self.nxy, (self.k1 + self.hi) * self.nxy)


def slab_of(nz, nxy, rank, world):
    base, extra = divmod(nz, world)
    k0 = rank * base + min(rank, extra)
    k1 = k0 + base + (1 if rank < extra else 0)
    return Slab(rank, world, k0, k1, 1 if k0 > 0 else 0, 1 if k1 < nz else 0, nxy)


def subgrid(g: W.GridDesc, slab: Slab) -> W.GridDesc:
    """The sub-grid of a slab: owned layers plus its ghost layers."""
    cells = slab.global_cells
    h = W.GridDesc(**{f: getattr(g, f) for f in g.__dataclass_fields__})
    h.nz = slab.k1 - slab.k0 + slab.lo + slab.hi
    h.top_depth = g.top_depth + (slab.k0 - slab.lo) * g.dz
    h.lnk = np.ascontiguousarray(g.lnk[cells])
    h.phi = np.ascontiguousarray(g.phi[cells])
    first = slab.k0 * slab.nxy
    last = slab.k1 * slab.nxy
    h.wells = []
    for w in g.wells:
        mine = [int(c) - (slab.k0 - slab.lo) * slab.nxy for c in w.cells if first <= int(c) < last]
        h.wells.append(W.Well(kind=w.kind, phase=w.phase, p_bh=w.p_bh, rw=w.rw, skin=w.skin,
                              cells=np.array(mine, dtype=np.int64)))
    return h


def exchange_ghosts(u: torch.Tensor, slab: Slab, group=None):
    """Fill the ghost layers of a variable-major sub-grid state u (nv, n_sub)
    from the neighbour ranks' owned boundary layers (in place)."""
    nxy, nl = slab.nxy, slab.k1 - slab.k0
    reqs = []
    lo_owned = u[:, slab.lo * nxy:(slab.lo + 1) * nxy].contiguous()
    hi_owned = u[:, (slab.lo + nl - 1) * nxy:(slab.lo + nl) * nxy].contiguous()
    lo_ghost = torch.empty_like(lo_owned)
    hi_ghost = torch.empty_like(hi_owned)
    if slab.lo:
        reqs.append(dist.isend(lo_owned, slab.rank - 1, group=group))
        reqs.append(dist.irecv(lo_ghost, slab.rank - 1, group=group))
    if slab.hi:
        reqs.append(dist.isend(hi_owned, slab.rank + 1, group=group))
        reqs.append(dist.irecv(hi_ghost, slab.rank + 1, group=group))
    for r in reqs:
        r.wait()
    if slab.lo:
        u[:, :nxy] = lo_ghost
    if slab.hi:
        u[:, (slab.lo + nl) * nxy:] = hi_ghost
    return u


def exchange_ghost_blocks(x: torch.Tensor, slab: Slab, nb: int, group=None):
    """Fill the ghost layers of a block-interleaved sub-grid vector x
    [n_sub * nb] (the layout of residuals and SpMV operands) in place."""
    exchange_ghosts(x.view(-1, nb).t(), slab, group)
    return x


def distributed_spmv(apply, x: torch.Tensor, slab: Slab, nb: int, group=None):
    """y = A x on a slab: the ghost layers of x are exchanged first, then
    ``apply`` (the sub-grid's block-CSR product, e.g. ``Grid.spmv``) runs on
    the whole sub-grid vector.  The owned rows of the result equal the same
    rows of the product on the whole grid: each owned row reads only owned and
    ghost cells, with the same blocks in the same order."""
    exchange_ghost_blocks(x, slab, nb, group)
    return apply(x)


def owned_rows(v: torch.Tensor, slab: Slab, nb: int):
    """The owned part of a block-interleaved sub-grid vector."""
    return v.view(-1, nb)[slab.owned]


def global_dot(a: torch.Tensor, b: torch.Tensor, group=None):
    """Sum over all ranks of the dot product of their owned parts (the
    Allreduce of the norms, Sec. 3.4.2)."""
    t = (a * b).sum().reshape(1).to(torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t[0]


def global_max(v: torch.Tensor, group=None):
    """Largest entry over all ranks (for the scaled-residual maxima)."""
    t = v.max().reshape(1).to(torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return t[0]


def block_jacobi(diag_blocks: torch.Tensor):
    """The block-Jacobi preconditioner of the owned rows: z = D^-1 r with D
    the owned cells' diagonal blocks (n_own, nb, nb); no communication."""
    inv = torch.linalg.inv(diag_blocks)

    def apply(r: torch.Tensor):
        nb = inv.shape[-1]
        return torch.einsum("cij,cj->ci", inv, r.view(-1, nb)).reshape(-1)
    return apply


def bicgstab(matvec, precond, b: torch.Tensor, x: torch.Tensor, dot, rtol: float, maxit: int):
    """Left-preconditioned BiCGSTAB on the owned part of the unknowns (the
    Krylov method of the linear solver, Sec. 3.3.3 and Sec. 5.1, with the
    block-Jacobi preconditioner the library's solver also uses):
    solves M^-1 A x = M^-1 b.  ``matvec(v)`` returns the owned rows of A v
    for owned v (a distributed product exchanges the ghost layers inside);
    ``precond`` applies M^-1 to owned rows; ``dot`` is the global dot product
    of owned vectors (an Allreduce across slabs).  With one domain these are
    the plain product and dot, so the partitioned iterates equal the
    single-domain ones up to the summation order of the dots.  Stops when
    ||M^-1 (b - A x)|| <= rtol ||M^-1 b|| or after maxit iterations.
    Returns (x, iterations, relative residual)."""
    r = precond(b - matvec(x))
    nb0 = float(torch.sqrt(dot(precond(b), precond(b))))
    r0 = r.clone()
    rho = alpha = omega = 1.0
    v = torch.zeros_like(b)
    p = torch.zeros_like(b)
    it = 0
    res = float(torch.sqrt(dot(r, r))) / (nb0 if nb0 > 0 else 1.0)
    while it < maxit and res > rtol:
        rho_new = float(dot(r0, r))
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = precond(matvec(p))
        alpha = rho_new / float(dot(r0, v))
        s = r - alpha * v
        t = precond(matvec(s))
        tt = float(dot(t, t))
        omega = float(dot(t, s)) / tt if tt > 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        it += 1
        res = float(torch.sqrt(dot(r, r))) / (nb0 if nb0 > 0 else 1.0)
    return x, it, res


def distributed_bicgstab(apply_sub, diag_blocks: torch.Tensor, b_own: torch.Tensor, x_own: torch.Tensor,
                         slab: Slab, nb: int, n_sub: int, rtol: float, maxit: int, group=None):
    """BiCGSTAB over slabs: ``apply_sub`` is the sub-grid's block-CSR product
    (its ghost rows are never used), ``diag_blocks`` the owned cells' diagonal
    blocks.  Each product first exchanges the ghost layers of its operand
    (point to point, Sec. 3.4.1); each dot product is an Allreduce of the
    owned parts (Sec. 3.4.2)."""
    full = torch.zeros(n_sub * nb, dtype=b_own.dtype)
    own = slice(slab.owned.start * nb, slab.owned.stop * nb)

    def matvec(v):
        full.zero_()
        full[own] = v
        y = distributed_spmv(apply_sub, full, slab, nb, group)
        return y[own].clone()

    return bicgstab(matvec, block_jacobi(diag_blocks), b_own, x_own,
                    lambda a, c: global_dot(a, c, group), rtol, maxit)
