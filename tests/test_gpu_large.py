"""A grid near the sizes the library is meant for: 600 x 600 x 100 three-phase
cells (36 million; 251 million blocks), linearised and multiplied by its
Jacobian once, with sampled rows of both recomputed by the oracle on their
windows (the product's rows from the oracle's blocks and the same vector)."""
import numpy as np
import pytest

from _gpu_common import RTOL_J, RTOL_R, RTOL_SPMV, assert_scaled_close, dev_state, need_gpu, window
from oracle.linearize import linearize
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_36m_cells_sampled_rows():
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    g, s = W.layered_box(seed=12, nx=600, ny=600, nz=100, frac_unsat=0.1)
    grid = ocp.Grid(g)
    assert grid.nnzb == 7 * g.N - 2 * (g.ny * g.nz + g.nx * g.nz + g.nx * g.ny)
    un, fn, uo, fo = dev_state(s)
    r, v, _ = grid.linearize(un, fn, uo, fo, s.dt)
    assert grid.status() == 0
    rp = grid.pattern()[0]
    rng = np.random.default_rng(13)
    cells = list(rng.choice(g.N, 60, replace=False)) + [0, g.N - 1, g.nx * g.ny * 50 + 300 * 600 + 300]
    cells += [int(w.cells[0]) for w in g.wells] + [int(w.cells[-1]) for w in g.wells]
    x = torch.as_tensor(rng.normal(size=3 * g.N), device="cuda")
    y = grid.spmv(v, x)
    for c in cells:
        h, st, centre = window(g, s, c)
        o = linearize(h, st.u_new, st.flag_new, st.u_old, st.flag_old, st.dt)
        a, b = int(rp[c]), int(rp[c + 1])
        assert_scaled_close(r[3 * c:3 * c + 3].cpu().numpy(), o["R"][centre], o["R_mag"][centre], RTOL_R,
                            "residual row %d" % c)
        oa, ob = o["row_ptr"][centre], o["row_ptr"][centre + 1]
        blocks = v[9 * a:9 * b].cpu().numpy().reshape(-1, 3, 3)
        assert_scaled_close(blocks, o["val"][oa:ob], o["val_mag"][oa:ob], RTOL_J, "jacobian row %d" % c)
        # the product's row from the oracle's own blocks and the same x entries
        cols = o["col_idx"][oa:ob]
        gcols = []
        for lc in cols:                      # window-local column -> global cell
            li, lj, lk = lc % h.nx, (lc // h.nx) % h.ny, lc // (h.nx * h.ny)
            ci, cj, ck = c % g.nx, (c // g.nx) % g.ny, c // (g.nx * g.ny)
                                             # the window starts one cell before c where it can
            i0, j0, k0 = max(ci - 1, 0), max(cj - 1, 0), max(ck - 1, 0)
            gcols.append((i0 + li) + g.nx * ((j0 + lj) + g.ny * (k0 + lk)))
        xs = x.view(-1, 3)[torch.as_tensor(gcols, device="cuda")].cpu().numpy()
        ref = np.einsum("sev,sv->e", o["val"][oa:ob], xs)
        mag = np.einsum("sev,sv->e", np.abs(o["val"][oa:ob]), np.abs(xs))
        assert_scaled_close(y[3 * c:3 * c + 3].cpu().numpy(), ref, mag, RTOL_SPMV + 4 * RTOL_J, "spmv row %d" % c)
