"""The slab partition on the GPU: each rank's sub-grid (owned layers plus
ghost layers holding the neighbours' primary variables), linearised by the
library, reproduces the owned rows of the whole grid's linearisation bit for
bit.  The ranks are emulated one after another on one GPU; their exchange is
covered by the gloo test."""
import numpy as np
import pytest

from _gpu_common import dev_state, need_gpu, torch
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 4])
def test_partitioned_linearization_is_bit_identical(world):
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    from paper_2406_10862_gb300 import partition as P
    g, s = W.layered_box(seed=9, nx=23, ny=17, nz=12, frac_unsat=0.2)
    full = ocp.Grid(g)
    r, v, ff = full.linearize(*dev_state(s), s.dt)
    rp = full.pattern()[0].cpu().numpy()
    r, v = r.cpu().numpy(), v.cpu().numpy()
    for rank in range(world):
        slab = P.slab_of(g.nz, g.nx * g.ny, rank, world)
        h = P.subgrid(g, slab)
        cells = slab.global_cells
        sub = W.State(u_new=s.u_new[:, cells], flag_new=s.flag_new[cells], u_old=s.u_old[:, cells],
                      flag_old=s.flag_old[cells], dt=s.dt)
        grid = ocp.Grid(h)
        rs, vs, _ = grid.linearize(*dev_state(sub), s.dt)
        assert grid.status() == 0
        rps = grid.pattern()[0].cpu().numpy()
        own = slab.owned
        gown = cells[own]
        assert np.array_equal(rs.cpu().numpy().reshape(-1, 3)[own], r.reshape(-1, 3)[gown])
        vs = vs.cpu().numpy().reshape(-1, 9)
        v9 = v.reshape(-1, 9)
        for lc, gc in zip(range(own.start, own.stop), gown):
            assert np.array_equal(vs[rps[lc]:rps[lc + 1]], v9[rp[gc]:rp[gc + 1]])


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_spmv_owned_rows_are_bit_identical(world):
    # each sub-grid's product with a vector whose ghost layers hold the
    # neighbours' entries reproduces the whole grid's owned rows bit for bit
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    from paper_2406_10862_gb300 import partition as P
    g, s = W.layered_box(seed=10, nx=19, ny=13, nz=9, frac_unsat=0.2)
    full = ocp.Grid(g)
    _, v, _ = full.linearize(*dev_state(s), s.dt)
    x = torch.as_tensor(np.random.default_rng(6).normal(size=3 * g.N), device="cuda")
    y = full.spmv(v, x).cpu().numpy().reshape(-1, 3)
    for rank in range(world):
        slab = P.slab_of(g.nz, g.nx * g.ny, rank, world)
        h = P.subgrid(g, slab)
        cells = slab.global_cells
        sub = W.State(u_new=s.u_new[:, cells], flag_new=s.flag_new[cells], u_old=s.u_old[:, cells],
                      flag_old=s.flag_old[cells], dt=s.dt)
        grid = ocp.Grid(h)
        _, vs, _ = grid.linearize(*dev_state(sub), s.dt)
        xs = x.view(-1, 3)[torch.as_tensor(cells, device="cuda")].reshape(-1).contiguous()
        ys = grid.spmv(vs, xs)
        got = P.owned_rows(ys, slab, 3).cpu().numpy()
        assert np.array_equal(got, y[cells[slab.owned]])
