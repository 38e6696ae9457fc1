"""Pins of the adaptive-coupling oracle (Sec. 4, steps 1-3) against hand-derived
cases, the strict threshold, the state semantics of the third variable, and an
independent graph construction whose components scipy finds."""
import importlib.util
import os
import shutil

import numpy as np
import pytest

import oracle.coupling as oracle_coupling
from paper_2406_10862_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _calm(nx, ny, nz, nphase=3):
    """A grid and a state pair with no change at all."""
    g, s = W.tiny(nx, ny, nz, nphase=nphase, seed=3, frac_unsat=0.0, wells=False)
    s.u_new[...] = s.u_old
    s.flag_new[...] = s.flag_old
    return g, s


def _run(C, g, s, px, py, pz, thr=5e-3):
    return C.coupling_components(g, s.u_new, s.flag_new, s.u_old, s.flag_old, thr, px, py, pz)


def pin_no_change_leaves_every_subdomain_alone(C):
    g, s = _calm(6, 6, 2)
    lab, marked, edges = _run(C, g, s, 3, 3, 2)
    assert not marked.any() and not edges
    assert np.array_equal(lab, np.arange(18))


def pin_box_split_is_near_equal_and_ordered(C):
    g, _ = _calm(7, 5, 3)
    sub = C.subdomains(g, 3, 2, 2)
    # along x, 7 cells in 3 parts: runs of 2, 2, 3 (floor(i * 3 / 7))
    assert sub[:7].tolist() == [0, 0, 0, 1, 1, 2, 2]
    # the last cell is in the last box
    assert sub[-1] == 3 * 2 * 2 - 1
    counts = np.bincount(sub)
    assert counts.min() >= 2 * 2 * 1 and counts.sum() == g.N


def pin_marked_interior_cell_couples_its_box_with_all_neighbours(C):
    # 9x9x1 grid in 3x3 boxes; the centre cell of the centre box (4) changes:
    # box 4 joins boxes 1, 3, 5 and 7 (its face neighbours), corners stay alone
    g, s = _calm(9, 9, 1)
    c = g.cell(4, 4, 0)
    s.u_new[1, c] += 0.01
    lab, marked, edges = _run(C, g, s, 3, 3, 1)
    assert marked.sum() == 1 and marked[c]
    assert lab.tolist() == [0, 1, 2, 1, 1, 1, 6, 1, 8]
    assert edges == {(1, 4), (3, 4), (4, 5), (4, 7)}


def pin_marked_cell_on_box_face(C):
    # cell (2, 1) is the last column of box 0; box 1 sees it as a ghost cell.
    # Rule (a) couples box 0 with boxes 1 and 3; rule (b) adds (0, 1) again.
    g, s = _calm(9, 9, 1)
    s.u_new[1, g.cell(2, 1, 0)] -= 0.01
    lab, _, edges = _run(C, g, s, 3, 3, 1)
    assert edges == {(0, 1), (0, 3)}
    assert lab.tolist() == [0, 0, 2, 0, 4, 5, 6, 7, 8]


def pin_gas_front_in_a_vertical_split(C):
    # one layer per box along z; gas rises in layers 0, 2 and 4: each of those
    # boxes joins the boxes above and below, which chains all six together
    g, s = _calm(4, 4, 6)
    for k in (0, 2, 4):
        s.u_new[2, g.cell(1, 1, k)] += 0.05
    lab, _, edges = _run(C, g, s, 1, 1, 6)
    assert edges == {(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)}
    assert np.all(lab == 0)


def pin_threshold_is_strict(C):
    # 0.25 -> 0.375 is exact in binary: a change of exactly 0.125
    g, s = _calm(4, 4, 1, nphase=2)
    s.u_old[1, :] = 0.25
    s.u_new[1, :] = 0.25
    s.u_new[1, 5] = 0.375
    assert not C.marked_cells(g, s.u_new, s.flag_new, s.u_old, s.flag_old, 0.125).any()
    m = C.marked_cells(g, s.u_new, s.flag_new, s.u_old, s.flag_old, np.nextafter(0.125, 0.0))
    assert m.sum() == 1 and m[5]


def pin_oil_saturation_counts_too(C):
    # water and gas each grow by 0.004 (below 0.005), so S_o = 1 - S_w - S_g
    # drops by 0.008: the oil saturation alone marks the cell
    g, s = _calm(3, 3, 1)
    s.u_new[1, 4] += 0.004
    s.u_new[2, 4] += 0.004
    m = C.marked_cells(g, s.u_new, s.flag_new, s.u_old, s.flag_old, 5e-3)
    assert m.sum() == 1 and m[4]


def pin_undersaturated_third_variable_is_not_a_saturation(C):
    # X = R_s in undersaturated cells: a large change of it marks nothing
    g, s = _calm(3, 3, 1)
    s.flag_old[:] = 1
    s.flag_new[:] = 1
    s.u_old[2, :] = 100.0
    s.u_new[2, :] = 150.0
    assert not C.marked_cells(g, s.u_new, s.flag_new, s.u_old, s.flag_old, 5e-3).any()
    # a saturated cell with S_g = 0.1 that becomes undersaturated loses its gas
    s.flag_old[7] = 0
    s.u_old[2, 7] = 0.1
    m = C.marked_cells(g, s.u_new, s.flag_new, s.u_old, s.flag_old, 5e-3)
    assert m.sum() == 1 and m[7]


def pin_everything_marked_is_one_component(C):
    g, s = _calm(5, 4, 3)
    s.u_new[1] += 0.1
    for parts in ((5, 4, 3), (2, 2, 2), (1, 4, 1)):
        lab, _, _ = _run(C, g, s, *parts)
        assert np.all(lab == 0)


def _min_labels(ncomp_labels):
    """Relabel a component labelling by the smallest member of each component."""
    out = np.empty_like(ncomp_labels)
    for c in np.unique(ncomp_labels):
        idx = np.flatnonzero(ncomp_labels == c)
        out[idx] = idx.min()
    return out


def pin_one_cell_per_subdomain_matches_star_graph_components(C):
    # with every cell its own subdomain, rule (a) joins each marked cell with
    # its face neighbours: the components are those of the union of the stars
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    g, s = W.tiny(6, 5, 4, seed=11, frac_unsat=0.3, wells=False)
    rng = np.random.default_rng(5)
    s.u_new[...] = s.u_old
    s.flag_new[...] = s.flag_old
    hit = rng.random(g.N) < 0.12
    s.u_new[1, hit] += 0.02
    lab, marked, _ = _run(C, g, s, g.nx, g.ny, g.nz)
    assert np.array_equal(marked, hit)
    rows, cols = [], []
    for c in np.flatnonzero(hit):
        i, j, k = c % g.nx, (c // g.nx) % g.ny, c // (g.nx * g.ny)
        for a, b, e in ((i + 1, j, k), (i - 1, j, k), (i, j + 1, k), (i, j - 1, k), (i, j, k + 1), (i, j, k - 1)):
            if 0 <= a < g.nx and 0 <= b < g.ny and 0 <= e < g.nz:
                rows.append(c)
                cols.append(g.cell(a, b, e))
    A = sp.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(g.N, g.N))
    _, comp = csg.connected_components(A, directed=False)
    assert np.array_equal(lab, _min_labels(comp))


def pin_components_match_scipy_on_fronts(C):
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    g, s = W.addm_2d(n=200)
    lab, marked, edges = _run(C, g, s, 20, 12, 1)
    assert 0 < marked.sum() < g.N // 10
    S = 240
    e = np.array(sorted(edges))
    A = sp.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(S, S))
    _, comp = csg.connected_components(A, directed=False)
    assert np.array_equal(lab, _min_labels(comp))
    # fronts around four separate injectors: four coupled regions
    u, cnt = np.unique(lab, return_counts=True)
    assert (cnt > 1).sum() == 4


PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__[4:])
def test_pin(pin):
    pin(oracle_coupling)


MUTATIONS = [
    ("change > threshold", "change >= threshold"),                          # strict threshold
    ("np.where(np.asarray(flag) == 0, u[2], 0.0)", "u[2]"),                  # R_s taken as S_g
    ("return [sw, 1.0 - sw - sg, sg]", "return [sw, sg]"),                   # oil dropped
    ("pick = rule_a | rule_b", "pick = rule_b"),                             # rule (a) dropped
    ("has_marked[sub[marked]] = True", "has_marked[marked[:len(has_marked)]] = True"),
    ("return (idx * parts) // n", "return (idx * parts + parts - 1) // n"),  # split rounding
    ("(i, nx, 1), (j, ny, nx)", "(i, nx, 1), (j, ny, ny)"),                  # wrong stride
    ("labels[w] = s", "labels[w] = v"),                                      # label not the root
]


@pytest.mark.parametrize("k", range(len(MUTATIONS)))
def test_planted_mistake_is_caught(tmp_path, k):
    old, new = MUTATIONS[k]
    dst = tmp_path / "oracle_cm"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst)
    f = dst / "coupling.py"
    src = f.read_text()
    assert src.count(old) == 1, old
    f.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("oracle_cm_coupling_%d" % k, f)
    C = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(C)
    failed = []
    for pin in PINS:
        try:
            pin(C)
        except (AssertionError, IndexError, ValueError):
            failed.append(pin.__name__)
    assert failed, "mutation %r passed every pin" % (old,)
