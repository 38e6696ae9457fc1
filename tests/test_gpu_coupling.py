"""GPU parity of the adaptive subdomain coupling (Sec. 4, steps 1-3): the
component labels and the number of marked cells must equal the oracle's
exactly, on hand-made cases, ragged box splits, one-cell subdomains, both
phase counts, and the 4000 x 4000 x 1 flood split over 1000 subdomains."""
import numpy as np
import pytest

from _gpu_common import dev_state, need_gpu
from oracle.coupling import coupling_components
from paper_2406_10862_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _both(g, s, thr, px, py, pz):
    need_gpu()
    from paper_2406_10862_gb300 import ocp
    grid = ocp.Grid(g)
    un, fn, uo, fo = dev_state(s)
    lab, work = grid.coupling_components(un, fn, uo, fo, thr, px, py, pz)
    S = px * py * pz
    w = work.cpu().numpy()
    ref, marked, _ = coupling_components(g, s.u_new, s.flag_new, s.u_old, s.flag_old, thr, px, py, pz)
    assert np.array_equal(lab.cpu().numpy().astype(np.int64), ref)
    assert w[2 * S] == int(marked.sum())
    assert 0 <= w[2 * S + 1] < max(S, 1)      # union-find retries
    assert w[2 * S + 2] == 0                   # no walk or retry bound reached
    grid.close()
    return ref


def _calm(nx, ny, nz, nphase=3):
    g, s = W.tiny(nx, ny, nz, nphase=nphase, seed=3, frac_unsat=0.0, wells=False)
    s.u_new[...] = s.u_old
    s.flag_new[...] = s.flag_old
    return g, s


def test_hand_cases():
    g, s = _calm(9, 9, 1)
    assert _both(g, s, 5e-3, 3, 3, 1).tolist() == list(range(9))
    s.u_new[1, g.cell(4, 4, 0)] += 0.01
    assert _both(g, s, 5e-3, 3, 3, 1).tolist() == [0, 1, 2, 1, 1, 1, 6, 1, 8]
    s.u_new[...] = s.u_old
    s.u_new[1, g.cell(2, 1, 0)] -= 0.01
    assert _both(g, s, 5e-3, 3, 3, 1).tolist() == [0, 0, 2, 0, 4, 5, 6, 7, 8]


def test_strict_threshold_and_oil():
    g, s = _calm(4, 4, 1, nphase=2)
    s.u_old[1, :] = 0.25
    s.u_new[1, :] = 0.25
    s.u_new[1, 5] = 0.375
    _both(g, s, 0.125, 2, 2, 1)
    _both(g, s, float(np.nextafter(0.125, 0.0)), 2, 2, 1)
    g, s = _calm(3, 3, 1)
    s.u_new[1, 4] += 0.004
    s.u_new[2, 4] += 0.004
    _both(g, s, 5e-3, 3, 3, 1)


@pytest.mark.parametrize("nphase", [2, 3])
@pytest.mark.parametrize("parts", [(1, 1, 1), (3, 2, 2), (7, 5, 3), (2, 5, 1)])
def test_fronts_on_ragged_splits(nphase, parts):
    g, _ = W.tiny(7, 5, 3, nphase=nphase, seed=21, wells=False)
    s = W.front_state(g, 9, [(1, 1, 1, 2.5, 2), (5, 3, 1, 1.5, 0)], width=0.6)
    _both(g, s, 5e-3, *parts)


@pytest.mark.parametrize("thr", [0.0, 1e-3, 5e-3, 0.03])
def test_thresholds_on_a_flood(thr):
    g, s = W.addm_2d(n=400)
    _both(g, s, thr, 40, 25, 1)


def test_one_cell_per_subdomain():
    g, _ = W.tiny(12, 10, 4, seed=5, wells=False)
    s = W.front_state(g, 6, [(6, 5, 2, 3.0, 2), (2, 2, 0, 2.0, 0)], width=0.8)
    _both(g, s, 5e-3, 12, 10, 4)


def test_full_size_flood_1000_subdomains():
    # the 16-million-cell two-dimensional flood split into 40 x 25 boxes
    g, s = W.addm_2d()
    ref = _both(g, s, 5e-3, 40, 25, 1)
    _, cnt = np.unique(ref, return_counts=True)
    assert (cnt > 1).sum() == 4


def test_near_threshold_and_special_values():
    # changes within a few ulps of the threshold (where the kernel's FP32
    # filter must defer to FP64), oil-only changes, huge, tiny, infinite and
    # NaN saturations: the marks must still equal the definition's
    g, s = _calm(20, 20, 4)
    rng = np.random.default_rng(17)
    N = g.N
    thr = 5e-3
    wo = rng.uniform(0.0, 0.8, N)
    go = rng.uniform(0.0, 0.1, N)
    s.u_old[1], s.u_old[2] = wo, go
    s.u_new[1], s.u_new[2] = wo.copy(), go.copy()
    q = N // 8
    # water change thr * (1 + O(1e-7)) and exact ulp steps around wo + thr
    s.u_new[1, :q] = wo[:q] + thr * (1.0 + rng.uniform(-1e-6, 1e-6, q))
    steps = np.arange(q) % 9 - 4
    base = wo[q:2 * q] + thr
    s.u_new[1, q:2 * q] = base + steps * np.spacing(base)
    # oil-only: water and gas each move by about thr / 2
    h = 0.5 * thr * (1.0 + rng.uniform(-1e-6, 1e-6, q))
    s.u_new[1, 2 * q:3 * q] = wo[2 * q:3 * q] + h
    s.u_new[2, 2 * q:3 * q] = go[2 * q:3 * q] + h
    # gas change near the threshold
    s.u_new[2, 3 * q:4 * q] = go[3 * q:4 * q] + thr * (1.0 + rng.uniform(-1e-6, 1e-6, q))
    # special values in either state
    special = [1e30, -1e30, 1e300, np.inf, -np.inf, np.nan, 1e-310, -1e-310, 1e-40, 3e38, 2.0 ** 127, 0.0]
    idx = np.arange(4 * q, 4 * q + 4 * len(special))
    for n, v in enumerate(special):
        s.u_new[1, idx[4 * n]] = v
        s.u_old[1, idx[4 * n + 1]] = v
        s.u_new[2, idx[4 * n + 2]] = v
        s.u_old[2, idx[4 * n + 3]] = v
    with np.errstate(invalid="ignore", over="ignore"):
        for t in (thr, 0.0, 1e-300, 0.5, 1e300):
            _both(g, s, t, 4, 5, 2)
    # the undersaturated third variable stays out of the test
    s.flag_new[::3] = 1
    s.flag_old[::3] = 1
    with np.errstate(invalid="ignore", over="ignore"):
        _both(g, s, thr, 4, 5, 2)


@pytest.mark.parametrize("parts", [(75, 80, 1), (100, 80, 1)])
def test_many_subdomains_shared_and_global_paths(parts):
    # 6000 subdomains still fit the shared-memory path, 8000 take the global one
    g, _ = W.tiny(100, 80, 1, seed=8, wells=False)
    fronts = [(30, 30, 0, 12.0, 2), (70, 50, 0, 9.0, 0), (20, 65, 0, 6.0, 0)]
    s = W.front_state(g, 12, fronts, width=1.0)
    _both(g, s, 5e-3, *parts)
