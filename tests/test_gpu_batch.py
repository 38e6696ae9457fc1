"""Batched ensemble: one pass over many uneven grids must equal linearising
each grid on its own, bit for bit, for every launch shape and in graph
replay; each model must also match the oracle."""
import numpy as np
import pytest

from _gpu_common import RTOL_J, RTOL_R, assert_scaled_close, dev_state, need_gpu, torch
from oracle.linearize import linearize as oracle_linearize
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (13, 7, 3), (31, 17, 5), (5, 40, 2), (64, 32, 4), (2, 3, 9)]


def ocp():
    need_gpu()
    from paper_2406_10862_gb300 import ocp as O
    O.load()
    return O


def build(O, nphase=3, seed=70):
    models = [W.tiny(*sh, nphase=nphase, seed=seed + k) for k, sh in enumerate(SHAPES)]
    grids = [O.Grid(g) for g, _ in models]
    ios = []
    for (g, s), grid in zip(models, grids):
        un, fn, uo, fo = dev_state(s)
        ios.append(dict(u_new=un, flag_new=fn, u_old=uo, flag_old=fo,
                        residual=torch.full((grid.nb * grid.N,), np.nan, dtype=torch.float64, device="cuda"),
                        bsr_val=torch.full((grid.nnzb * grid.nb ** 2,), np.nan, dtype=torch.float64, device="cuda"),
                        face_flux=torch.full((3 * grid.nb * grid.N,), np.nan, dtype=torch.float64, device="cuda")))
    return models, grids, ios


def per_model(grids, models, ios, dt):
    out = []
    for grid, (g, s), io in zip(grids, models, ios):
        r, v, f = grid.linearize(io["u_new"], io["flag_new"], io["u_old"], io["flag_old"], dt, want_face_flux=True)
        out.append((r.clone(), v.clone(), f.clone()))
    return out


def same_bits(a, b):
    return torch.equal(a.view(torch.int64), b.view(torch.int64))


@pytest.mark.parametrize("nphase", [3, 2])
def test_batch_equals_per_model_bitwise_for_every_shape(nphase):
    O = ocp()
    models, grids, ios = build(O, nphase)
    ref = per_model(grids, models, ios, 1.0)
    batch = O.Batch(grids)
    batch.set_io(ios)
    shapes = [dict(cells_per_tile=[256, 256, 256], ctas_per_sm=[0, 0, 0]),
              dict(cells_per_tile=[128, 256, 128], ctas_per_sm=[1, 2, 4]),
              dict(cells_per_tile=[256, 128, 256], ctas_per_sm=[8, 1, 16]),
              dict(cells_per_tile=[32, 64, 32], ctas_per_sm=[0, 3, 0]),
              # ordered (persistent) launches: face + assembly, then cell + face + assembly
              dict(cells_per_tile=[128, 128, 256], ctas_per_sm=[0, 0, 0], ordered=1),
              dict(cells_per_tile=[64, 32, 256], ctas_per_sm=[2, 1, 0], ordered=1),
              dict(cells_per_tile=[128, 128, 256], ctas_per_sm=[0, 0, 0], ordered=2),
              dict(cells_per_tile=[128, 256, 128], ctas_per_sm=[0, 1, 0], ordered=2),
              dict(cells_per_tile=[128, 32, 128], ctas_per_sm=[0, 2, 0], ordered=2),
              dict(cells_per_tile=[64, 32, 32], ctas_per_sm=[0, 0, 0], ordered=3),
              dict(cells_per_tile=[32, 32, 32], ctas_per_sm=[1, 2, 1], ordered=3)]
    for k, sh in enumerate(shapes):
        batch.set_shape(sh)
        for io in ios:
            io["residual"].fill_(np.nan)
            io["bsr_val"].fill_(np.nan)
            io["face_flux"].fill_(np.nan)
        batch.linearize(1.0, graph=(k in (2, 6)))
        assert batch.status() == 0
        for io, (r, v, f) in zip(ios, ref):
            assert same_bits(io["residual"], r) and same_bits(io["bsr_val"], v) and same_bits(io["face_flux"], f)


def test_batch_graph_replay_and_dt_change():
    O = ocp()
    models, grids, ios = build(O, 3, seed=80)
    batch = O.Batch(grids)
    batch.set_io(ios)
    for dt in (1.0, 0.25, 0.25, 3.0):
        batch.linearize(dt, graph=True)
        torch.cuda.synchronize()
        got = [(io["residual"].clone(), io["bsr_val"].clone()) for io in ios]
        ref = per_model(grids, models, ios, dt)
        for (r, v), (r0, v0, f0) in zip(got, ref):
            assert same_bits(r, r0) and same_bits(v, v0)


def test_batch_models_match_the_oracle():
    O = ocp()
    models, grids, ios = build(O, 3, seed=90)
    batch = O.Batch(grids)
    batch.set_io(ios)
    batch.linearize(0.5)
    assert batch.status() == 0
    for (g, s), io in zip(models, ios):
        o = oracle_linearize(g, s.u_new, s.flag_new, s.u_old, s.flag_old, 0.5)
        assert_scaled_close(io["residual"].cpu().numpy(), o["R"], o["R_mag"], RTOL_R, "batched residual")
        assert_scaled_close(io["bsr_val"].cpu().numpy(), o["val"], o["val_mag"], RTOL_J, "batched jacobian")


def test_tuner_returns_a_valid_shape_and_keeps_results():
    O = ocp()
    models, grids, ios = build(O, 3, seed=100)
    ref = per_model(grids, models, ios, 1.0)
    batch = O.Batch(grids)
    batch.set_io(ios)
    best = batch.tune(1.0, reps=2)
    assert all(t in (32, 64, 128, 256) for t in best["cells_per_tile"])
    assert all(0 <= c <= 16 for c in best["ctas_per_sm"]) and best["ordered"] in (0, 1, 2, 3)   # not 4: 6 models
    assert batch.get_shape() == best
    batch.linearize(1.0, graph=True)
    torch.cuda.synchronize()
    for io, (r, v, f) in zip(ios, ref):
        assert same_bits(io["residual"], r) and same_bits(io["bsr_val"], v)


def test_batch_status_and_errors():
    O = ocp()
    models, grids, ios = build(O, 3, seed=110)
    batch = O.Batch(grids)
    with pytest.raises(O.OcpError):
        batch.linearize(1.0)                       # no io yet
    ios[3]["u_new"][7] = float("nan")
    batch.set_io(ios)
    batch.linearize(1.0)
    assert batch.status() == O.OCP_ERR_NONFINITE
    assert batch.status() == 0
    g2, _ = W.tiny(3, 3, 3, nphase=2, seed=1)
    with pytest.raises(O.OcpError):
        O.Batch([grids[0], O.Grid(g2)])            # mixed block sizes
    with pytest.raises(O.OcpError):
        batch.set_shape(dict(cells_per_tile=[48, 256, 256], ctas_per_sm=[0, 0, 0]))
    with pytest.raises(O.OcpError):                 # one cluster takes one grid only
        batch.set_shape(dict(cells_per_tile=[64, 256, 256], ctas_per_sm=[0, 0, 0], ordered=4))
    with pytest.raises(O.OcpError):
        batch.set_shape(dict(cells_per_tile=[64, 256, 256], ctas_per_sm=[0, 0, 0], ordered=5))


def test_one_grid_batch_runs_as_one_cluster():
    """A batch of one small grid starts in the one-cluster launch; set, tuned,
    or replayed as a graph across dt changes, it gives the bits of the grid's
    own three plain launches."""
    O = ocp()
    g, s = W.tiny(10, 10, 3, nphase=3, seed=120, frac_unsat=0.3)
    grid = O.Grid(g)
    un, fn, uo, fo = dev_state(s)
    io = dict(u_new=un, flag_new=fn, u_old=uo, flag_old=fo,
              residual=torch.empty(grid.nb * grid.N, dtype=torch.float64, device="cuda"),
              bsr_val=torch.empty(grid.nnzb * grid.nb ** 2, dtype=torch.float64, device="cuda"),
              face_flux=torch.empty(3 * grid.nb * grid.N, dtype=torch.float64, device="cuda"))
    batch = O.Batch([grid])
    batch.set_io([io])
    assert batch.get_shape()["ordered"] == 4
    grid.set_shape(dict(cells_per_tile=[128, 128, 256], ctas_per_sm=[0, 0, 0], ordered=0))
    for dt in (1.0, 0.25, 0.25, 3.0):
        r, v, f = (t.clone() for t in grid.linearize(un, fn, uo, fo, dt, want_face_flux=True))
        for graph in (False, True):
            for k in ("residual", "bsr_val", "face_flux"):
                io[k].fill_(np.nan)
            batch.linearize(dt, graph=graph)
            torch.cuda.synchronize()
            assert batch.status() == 0
            assert same_bits(io["residual"], r) and same_bits(io["bsr_val"], v) and same_bits(io["face_flux"], f)
    best = batch.tune(1.0, reps=2)
    assert best["ordered"] in (0, 1, 2, 3, 4)
    batch.linearize(1.0)
    torch.cuda.synchronize()
    r, v, f = grid.linearize(un, fn, uo, fo, 1.0, want_face_flux=True)
    assert same_bits(io["residual"], r) and same_bits(io["bsr_val"], v)
