"""Multi-rank path on the CPU (gloo, world size 2 and 3): a slab partition of
one grid with ghost layers filled by point-to-point exchange of primary
variables must reproduce, bit for bit, the owned rows of the unpartitioned
linearisation (the invariance the paper shows as identical Newton iteration
counts for every process count in its scaling study).  The rows are computed
by the oracle on each rank's sub-grid; the GPU library computes the same rows
in the same order."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.linearize import linearize
        from paper_2406_10862_gb300 import partition as P
        from paper_2406_10862_gb300 import workloads as W
        g, s = W.tiny(5, 4, 7, seed=77, frac_unsat=0.3)
        slab = P.slab_of(g.nz, g.nx * g.ny, rank, world)
        h = P.subgrid(g, slab)
        cells = slab.global_cells
        own = slab.owned
        # each rank starts from its owned layers only; ghosts arrive by exchange
        u_new = torch.zeros((g.nphase, len(cells)), dtype=torch.float64)
        u_old = torch.zeros_like(u_new)
        f_new = torch.full((len(cells),), -1, dtype=torch.int8)
        f_old = torch.full_like(f_new, -1)
        gown = cells[own]
        u_new[:, own] = torch.from_numpy(s.u_new[:, gown])
        u_old[:, own] = torch.from_numpy(s.u_old[:, gown])
        f_new[own] = torch.from_numpy(s.flag_new[gown])
        f_old[own] = torch.from_numpy(s.flag_old[gown])
        P.exchange_ghosts(u_new, slab)
        P.exchange_ghosts(u_old, slab)
        P.exchange_ghosts(f_new.view(1, -1), slab)
        P.exchange_ghosts(f_old.view(1, -1), slab)
        o = linearize(h, u_new.numpy(), f_new.numpy(), u_old.numpy(), f_old.numpy(), s.dt)
        rp = o["row_ptr"]
        rows = range(own.start, own.stop)
        blocks = np.concatenate([o["val"][rp[r]:rp[r + 1]] for r in rows])
        out_q.put((rank, gown, o["R"][own], blocks, float(o["well_rate"].sum())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_rows_are_bit_identical(world):
    from oracle.linearize import linearize
    from paper_2406_10862_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g, s = W.tiny(5, 4, 7, seed=77, frac_unsat=0.3)
    full = linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt)
    rp = full["row_ptr"]
    seen = np.zeros(g.N, dtype=bool)
    well_total = 0.0
    for rank, gown, R, blocks, wsum in sorted(res, key=lambda t: t[0]):
        assert np.array_equal(R, full["R"][gown])
        ref = np.concatenate([full["val"][rp[c]:rp[c + 1]] for c in gown])
        assert np.array_equal(blocks, ref)
        seen[gown] = True
        well_total += wsum
    assert seen.all()
    assert well_total == pytest.approx(float(full["well_rate"].sum()), rel=1e-13)


def _spmv_worker(rank, world, port, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.linearize import linearize
        from oracle.spmv import bsr_spmv
        from paper_2406_10862_gb300 import partition as P
        from paper_2406_10862_gb300 import workloads as W
        g, s = W.tiny(4, 5, 8, seed=78, frac_unsat=0.3)
        nb = g.nphase
        slab = P.slab_of(g.nz, g.nx * g.ny, rank, world)
        h = P.subgrid(g, slab)
        cells = slab.global_cells
        own = slab.owned
        # the sub-grid's Jacobian from the exchanged state (as above)
        o = linearize(h, s.u_new[:, cells], s.flag_new[cells], s.u_old[:, cells], s.flag_old[cells], s.dt)
        x_glob = np.random.default_rng(5).normal(size=(g.N, nb))
        x = torch.zeros((len(cells), nb), dtype=torch.float64)
        x[own] = torch.from_numpy(x_glob[cells[own]])           # owned part only; ghosts arrive by exchange
        apply = lambda v: torch.from_numpy(
            bsr_spmv(o["row_ptr"], o["col_idx"], o["val"], v.numpy().ravel())[0].copy())
        y = P.distributed_spmv(apply, x.view(-1), slab, nb)
        y_own = P.owned_rows(y, slab, nb).numpy().copy()
        d = P.global_dot(P.owned_rows(y, slab, nb), P.owned_rows(y, slab, nb))
        m = P.global_max(P.owned_rows(y, slab, nb).abs())
        out_q.put((rank, cells[own], y_own, float(d), float(m)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_spmv_rows_and_norms(world):
    from oracle.linearize import linearize
    from oracle.spmv import bsr_spmv
    from paper_2406_10862_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_spmv_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g, s = W.tiny(4, 5, 8, seed=78, frac_unsat=0.3)
    o = linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt)
    x = np.random.default_rng(5).normal(size=(g.N, g.nphase))
    y = bsr_spmv(o["row_ptr"], o["col_idx"], o["val"], x.ravel())[0].reshape(-1, g.nphase)
    seen = np.zeros(g.N, dtype=bool)
    for rank, gown, y_own, d, m in res:
        assert np.array_equal(y_own, y[gown])          # owned rows bit for bit
        assert d == pytest.approx(float((y * y).sum()), rel=1e-13)
        assert m == float(np.abs(y).max())
        seen[gown] = True
    assert seen.all()


def _solver_worker(rank, world, port, out_q, maxit):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.linearize import linearize
        from oracle.spmv import bsr_spmv
        from paper_2406_10862_gb300 import partition as P
        from paper_2406_10862_gb300 import workloads as W
        g, s = W.tiny(4, 3, 8, seed=79, frac_unsat=0.3)
        nb = g.nphase
        slab = P.slab_of(g.nz, g.nx * g.ny, rank, world)
        h = P.subgrid(g, slab)
        cells = slab.global_cells
        own = slab.owned
        o = linearize(h, s.u_new[:, cells], s.flag_new[cells], s.u_old[:, cells], s.flag_old[cells], s.dt)
        apply = lambda v: torch.from_numpy(
            bsr_spmv(o["row_ptr"], o["col_idx"], o["val"], v.numpy())[0].copy())
        rp, ci = o["row_ptr"], o["col_idx"]
        diag = torch.from_numpy(np.stack([o["val"][rp[c] + np.nonzero(ci[rp[c]:rp[c + 1]] == c)[0][0]]
                                          for c in range(own.start, own.stop)]))
        b = torch.from_numpy(-o["R"][own].ravel().copy())
        x, it, res = P.distributed_bicgstab(apply, diag, b, torch.zeros_like(b), slab, nb, len(cells), 0.0,
                                            maxit)
        out_q.put((rank, cells[own], x.numpy().copy(), it, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,maxit", [(2, 6), (2, 200), (3, 6)])
def test_distributed_bicgstab_follows_the_single_domain_iterates(world, maxit):
    """Block-Jacobi BiCGSTAB over slabs (ghost layers of every operand
    exchanged point to point, every dot product an Allreduce) takes the same
    iterates as the single-domain solver to rounding (only the dots sum in
    another order), after a few iterations and at convergence."""
    from oracle.linearize import linearize
    from oracle.spmv import bsr_spmv
    from paper_2406_10862_gb300 import partition as P
    from paper_2406_10862_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solver_worker, args=(r, world, port, q, maxit)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g, s = W.tiny(4, 3, 8, seed=79, frac_unsat=0.3)
    nb = g.nphase
    o = linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, s.dt)
    rp, ci = o["row_ptr"], o["col_idx"]
    diag = torch.from_numpy(np.stack([o["val"][rp[c] + np.nonzero(ci[rp[c]:rp[c + 1]] == c)[0][0]]
                                      for c in range(g.N)]))
    matvec = lambda v: torch.from_numpy(bsr_spmv(rp, ci, o["val"], v.numpy())[0].copy())
    b = torch.from_numpy(-o["R"].ravel().copy())
    x_ref, it_ref, res_ref = P.bicgstab(matvec, P.block_jacobi(diag), b, torch.zeros_like(b),
                                        lambda a, c: (a * c).sum(), 0.0, maxit)
    x_ref = x_ref.numpy().reshape(-1, nb)
    seen = np.zeros(g.N, dtype=bool)
    scale = np.abs(x_ref).max(axis=0)
    for rank, gown, x, it, r in res:
        assert it == it_ref
        assert np.all(np.abs(x.reshape(-1, nb) - x_ref[gown]) <= 1e-9 * scale)
        seen[gown] = True
    assert seen.all()
    if maxit > 100:
        assert res_ref < 1e-12
        # the converged iterate solves the system
        A = np.zeros((g.N * nb, g.N * nb))
        for r_ in range(g.N):
            for k in range(rp[r_], rp[r_ + 1]):
                A[r_ * nb:(r_ + 1) * nb, ci[k] * nb:(ci[k] + 1) * nb] = o["val"][k]
        xs = np.linalg.solve(A, b.numpy())
        assert np.allclose(x_ref.ravel(), xs, rtol=1e-8, atol=1e-10 * np.abs(xs).max())
