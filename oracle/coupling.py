"""Adaptive coupling of subdomains, written out plainly (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The adaptively coupled domain decomposition of Sec. 4 decides at the start of
every time step which subdomains to solve together:
  1. mark the cells whose phase saturation changed by more than a threshold
     over the previous step (the paper uses 5e-3);
  2. build a coupling graph between subdomains: (a) a subdomain with a marked
     interior cell is coupled with every neighbouring subdomain; (b) a
     subdomain with a marked ghost cell is coupled with the subdomain that
     owns that cell;
  3. take the connected components of the graph.
Subdomains here are the boxes of a px x py x pz split of the grid (the paper
partitions with ParMetis); a subdomain's ghost cells are the cells of other
subdomains that share a face with one of its cells.  Components are labelled
by their smallest subdomain index.
"""
from __future__ import annotations

import numpy as np


def box_of(n, parts, idx):
    """Part of index idx when n cells are split into `parts` near-equal runs."""
    return (idx * parts) // n


def subdomains(spec, px, py, pz):
    nx, ny, nz = int(spec.nx), int(spec.ny), int(spec.nz)
    c = np.arange(nx * ny * nz)
    i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
    return box_of(nx, px, i) + px * (box_of(ny, py, j) + py * box_of(nz, pz, k))


def saturations(spec, u, flag):
    u = np.asarray(u, dtype=np.float64).reshape(int(spec.nphase), -1)
    sw = u[1]
    if spec.nphase == 3:
        sg = np.where(np.asarray(flag) == 0, u[2], 0.0)
        return [sw, 1.0 - sw - sg, sg]
    return [sw, 1.0 - sw]


def marked_cells(spec, u_new, flag_new, u_old, flag_old, threshold):
    """Step 1: cells where some phase saturation moved by more than threshold."""
    sn = saturations(spec, u_new, flag_new)
    so = saturations(spec, u_old, flag_old)
    change = np.max(np.abs(np.stack(sn) - np.stack(so)), axis=0)
    return change > threshold


def face_pairs(spec):
    """Every ordered pair (c, n) of cells sharing a face, as two index arrays."""
    nx, ny, nz = int(spec.nx), int(spec.ny), int(spec.nz)
    c = np.arange(nx * ny * nz)
    i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
    lo = []
    hi = []
    for q, n, stride in ((i, nx, 1), (j, ny, nx), (k, nz, nx * ny)):
        a = c[q < n - 1]
        lo += [a, a + stride]
        hi += [a + stride, a]
    return np.concatenate(lo), np.concatenate(hi)


def coupling_components(spec, u_new, flag_new, u_old, flag_old, threshold, px, py, pz):
    """Steps 1-3.  Returns (labels per subdomain, marked cells, edge set)."""
    S = px * py * pz
    sub = subdomains(spec, px, py, pz)
    marked = marked_cells(spec, u_new, flag_new, u_old, flag_old, threshold)
    # faces between different subdomains: c's subdomain sees n as a ghost cell
    c, n = face_pairs(spec)
    cross = sub[c] != sub[n]
    c, n = c[cross], n[cross]
    s_of, t_of = sub[c], sub[n]
    has_marked = np.zeros(S, dtype=bool)
    has_marked[sub[marked]] = True
    rule_a = has_marked[s_of]          # (a) s holds a marked interior cell
    rule_b = marked[n]                 # (b) s holds the marked ghost cell n, owned by t
    pick = rule_a | rule_b
    lo = np.minimum(s_of[pick], t_of[pick])
    hi = np.maximum(s_of[pick], t_of[pick])
    edges = set(zip(lo.tolist(), hi.tolist()))
    # step 3: connected components by depth-first search
    adj = [[] for _ in range(S)]
    for s, t in edges:
        adj[s].append(t)
        adj[t].append(s)
    labels = np.full(S, -1, dtype=np.int64)
    for s in range(S):
        if labels[s] >= 0:
            continue
        labels[s] = s
        stack = [s]
        while stack:
            v = stack.pop()
            for w in adj[v]:
                if labels[w] < 0:
                    labels[w] = s
                    stack.append(w)
    return labels, marked, edges
