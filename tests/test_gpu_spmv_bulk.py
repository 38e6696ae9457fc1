"""The two block-CSR product kernels for 2x2 and 1x1 blocks give identical
bits.  When the matrix is 16-byte aligned, the library stages each CTA's
slice of it in shared memory with one bulk asynchronous copy.  Otherwise it
reads the blocks straight into registers.  A copy of the matrix shifted by
one double forces the second path.  The 2x2 products run through
``ocp_bsr_spmv``, with and without alpha and beta, from one cell up to the
1.12 M-cell oil-water model.  The 1x1 products run inside the scalar
BiCGSTAB of the IMPEC pressure system, on a matrix of odd size whose last
double lies past the copy's 16-byte end."""
import numpy as np
import pytest

from _gpu_common import dev_state, need_gpu
from oracle.pn import natural_to_pn
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def shifted(t):
    """The same values at an address 8 bytes past a 16-byte boundary."""
    buf = torch.empty(t.numel() + 1, dtype=t.dtype, device=t.device)
    v = buf[1:]
    v.copy_(t)
    assert v.data_ptr() % 16 == 8
    return v


def _grid(g):
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    return ocp.Grid(g)


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.7, 0.3)])
@pytest.mark.parametrize("case", ["1x1x1", "33x2x2", "17x9x2", "channelised 60x220x85"])
def test_two_by_two_paths_agree(case, alpha, beta):
    if case.startswith("channelised"):
        g, s = W.channelised_ow()
    else:
        nx, ny, nz = (int(a) for a in case.split("x"))
        g, s = W.tiny(nx, ny, nz, nphase=2, seed=nx + ny + nz)
    grid = _grid(g)
    un, fn, uo, fo = dev_state(s)
    _, val, _ = grid.linearize(un, fn, uo, fo, s.dt)
    assert val.data_ptr() % 16 == 0
    rng = np.random.default_rng(5)
    x = torch.as_tensor(rng.normal(size=2 * g.N), device="cuda")
    y0 = torch.as_tensor(rng.normal(size=2 * g.N), device="cuda")
    y_bulk = grid.spmv(val, x, alpha, beta, y0.clone())
    y_reg = grid.spmv(shifted(val), x, alpha, beta, y0.clone())
    assert grid.status() == 0
    assert torch.equal(y_bulk, y_reg)


@pytest.mark.parametrize("nphase", [3, 2])
def test_scalar_solver_paths_agree(nphase):
    g, s = W.tiny(5, 3, 3, nphase=nphase, seed=31, frac_unsat=0.3 if nphase == 3 else 0.0, rs_hi=0.7)
    assert (7 * g.N - 2 * (g.ny * g.nz + g.nx * g.nz + g.nx * g.ny)) * 8 % 16 == 8   # odd-sized matrix
    grid = _grid(g)
    pn = torch.as_tensor(np.ascontiguousarray(natural_to_pn(g, s.u_new, s.flag_new).ravel()), device="cuda")
    val, rhs = grid.impec_pressure(pn, 0.5)
    out = []
    for v in (val, shifted(val)):
        dp = torch.zeros(g.N, dtype=torch.float64, device="cuda")
        st, it, rr = grid.bicgstab_scalar(v, rhs, dp, 1e-13, 500)
        out.append((dp, it, rr))
    assert grid.status() == 0
    assert torch.equal(out[0][0], out[1][0]) and out[0][1] == out[1][1] and out[0][2] == out[1][2]
