"""Nested dissection of a general graph with vertex coordinates (Sec. 3.1, Alg. 1).

Test infrastructure (the oracle): the library's `spalu_nd_order_csr` is checked against it.
Each subgraph is cut by the separator walk of Sec. 3.1 (centre vertex nearest the coordinate
median, direction +x when the bounding box is narrower than tall, else +y, walks maximising
D(u, v, c, d) of Eq. (degreebias) with theta = 0.1 in +d and -d), the rest splits into the
two sides of the separator, and both sides are dissected again until a part has at most
`leaf_size` vertices.

Readings (the paper is silent on these points):
  * A walk ends where D <= 0 (Sec. 3.1), where no unvisited neighbour is left, or at the
    first vertex on the subgraph's boundary (a vertex with a neighbour outside the subgraph,
    or on the domain's boundary: the caller's mask, by default the vertices with fewer
    neighbours than the graph's most connected one, which is the boundary of a grid): on a
    grid the second term of D stays positive along an edge, so the walk would otherwise
    follow it.
  * Values of D within 1e-12 of each other count as equal and the first neighbour in
    adjacency order wins; D <= 1e-12 stops the walk; the centre is the first vertex within
    1e-12 (relative) of the smallest squared distance to the median.  These tolerances make
    the choice independent of the rounding of one implementation or another.
  * The sides: the vertices of the part not in the separator form connected components; a
    component goes to the first side when its first vertex (lowest id) lies below the line
    through the centre along d (smaller coordinate across d), else to the second.  A part
    whose separator leaves one side empty is a leaf.
  * Order I (Sec. 2.2 puts separators after the subgraphs): every leaf's vertices in
    increasing id, leaves in depth-first order (first side first), then the separators by
    level L..1, depth-first within a level, each in walk order (from the -d end to the +d end).
On a regular grid with leaf_size = 225 this is the grid dissection of `oracle.nd` (tested).
"""
from __future__ import annotations

import math

import numpy as np

THETA = 0.1
TOL = 1e-12


def _walk(coords, nbrs, inpart, boundary, c, d, taken=()):
    path, v, seen = [], c, {c, *taken}
    while True:
        best, bestu = None, None
        for u in nbrs[v]:
            if not inpart[u] or u in seen:
                continue
            a = coords[u] - coords[v]
            b = coords[u] - coords[c]
            na = math.sqrt(a[0] * a[0] + a[1] * a[1])
            nb = math.sqrt(b[0] * b[0] + b[1] * b[1])
            t1 = (a[0] * d[0] + a[1] * d[1]) / na
            t2 = 0.0 if nb == 0.0 else (b[0] * d[0] + b[1] * d[1]) / nb
            val = t1 + THETA * t2
            if best is None or val > best + TOL:
                best, bestu = val, u
        if bestu is None or best <= TOL:
            return path
        path.append(bestu)
        seen.add(bestu)
        if boundary[bestu]:
            return path
        v = bestu


def nested_dissection_graph(coords, indptr, indices, leaf_size: int, domain_boundary=None):
    """Returns (perm, level): perm = order I, level[v] = 0 for a leaf vertex, else the level
    (1 = the first cut) of the separator holding v.  domain_boundary: optional boolean mask of
    the vertices on the domain's boundary."""
    coords = np.asarray(coords, dtype=np.float64)
    n = coords.shape[0]
    nbrs = [[int(u) for u in indices[indptr[v]:indptr[v + 1]] if u != v] for v in range(n)]
    maxdeg = max((len(a) for a in nbrs), default=0)
    if domain_boundary is None:
        domain_boundary = np.array([len(a) < maxdeg for a in nbrs], dtype=bool)
    level = np.zeros(n, dtype=np.int64)
    leaves, seps = [], {}

    def rec(part, l):
        part = sorted(part)
        if len(part) <= leaf_size:
            leaves.append(part)
            return
        inpart = np.zeros(n, dtype=bool)
        inpart[part] = True
        P = coords[part]
        med = np.array([np.median(P[:, 0]), np.median(P[:, 1])])
        d2 = (P[:, 0] - med[0]) ** 2 + (P[:, 1] - med[1]) ** 2
        dmin = d2.min()
        c = part[int(np.nonzero(d2 <= dmin + TOL * max(dmin, 1.0))[0][0])]
        width = P[:, 0].max() - P[:, 0].min()
        height = P[:, 1].max() - P[:, 1].min()
        d = (1.0, 0.0) if width < height else (0.0, 1.0)
        boundary = np.zeros(n, dtype=bool)
        for v in part:
            boundary[v] = bool(domain_boundary[v]) or any(not inpart[u] for u in nbrs[v])
        fwd = _walk(coords, nbrs, inpart, boundary, c, d)
        bwd = _walk(coords, nbrs, inpart, boundary, c, (-d[0], -d[1]), fwd)   # fwd's vertices are taken
        sep = bwd[::-1] + [c] + fwd
        insep = set(sep)
        # components of the rest
        rest = [v for v in part if v not in insep]
        comp = {}
        sides = ([], [])
        across = 1 if d[0] == 1.0 else 0          # the coordinate across the separator
        for v in rest:
            if v in comp:
                continue
            stack, members = [v], []
            comp[v] = True
            while stack:
                x = stack.pop()
                members.append(x)
                for u in nbrs[x]:
                    if inpart[u] and u not in insep and u not in comp:
                        comp[u] = True
                        stack.append(u)
            first = min(members)
            side = 0 if coords[first][across] < coords[c][across] else 1
            sides[side].extend(members)
        if not sides[0] or not sides[1]:
            leaves.append(part)
            return
        for v in sep:
            level[v] = l
        seps.setdefault(l, []).append(sep)
        rec(sides[0], l + 1)
        rec(sides[1], l + 1)

    rec(list(range(n)), 1)
    order = [v for leaf in leaves for v in leaf]
    for l in sorted(seps, reverse=True):
        for sep in seps[l]:
            order.extend(sep)
    return np.array(order, dtype=np.int64), level
