"""Nested dissection of a regular grid with segment information (Sec. 2.2, Sec. 3, Alg. 1).

Readings of the paper used here (each is a documented choice, not a quotation):
  * Separator of a box (Sec. 3.1): the separating direction is the x axis when the box is
    narrower than it is tall, else the y axis; on a grid box with odd sides the median
    centre and the degree-bias walk of Eq. (degreebias) with theta=0.1 give the straight
    middle line (``separator_walk`` restates the walk literally and the tests check this).
  * Recursion stops at leaf boxes of ``leaf x leaf`` interior nodes (leaf=15: a 16x16 pitch
    with 1-wide separators).  Separators created while cutting depth-(l-1) boxes are the
    level-l separators; leaves are the depth-L boxes ("level L+1" in Sec. 4.3).
  * Order I (Sec. 2.2 puts separators after the subgraphs and eliminates leaves first):
    all leaf interiors (leaves in depth-first order, lower/left child first; inside a leaf
    x fastest), then separators level L, L-1, ..., 1; inside a level in depth-first order
    of the boxes they cut; inside a separator by increasing coordinate.
  * Segments at level l (Sec. 2.3.1, Sec. 3.2): every side of a depth-l box between two
    corners is a regular segment; every interior crossing of separator lines that is a
    corner of a depth-l box is a junction.  Sides on the Dirichlet boundary do not exist.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Box:
    x0: int
    x1: int
    y0: int
    y1: int
    depth: int

    @property
    def w(self):
        return self.x1 - self.x0 + 1

    @property
    def h(self):
        return self.y1 - self.y0 + 1


@dataclass
class Segment:
    key: tuple            # ('H', y, xa, xb) or ('V', x, ya, yb): geometric extent (inclusive)
    level: int
    sid: int              # index used to key the random stream (see philox.py)
    nodes: np.ndarray     # grid nodes of the side in increasing coordinate
    boxes: list           # the (one or two) depth-l boxes having this side
    is_separator: bool    # True when it is a level-l separator


@dataclass
class Level:
    level: int
    boxes: list                    # depth-l boxes, depth-first order
    segments: dict                 # key -> Segment
    corners: list                  # grid nodes of junctions (corners of depth-l boxes)
    separators: list               # keys of level-l separators, depth-first order of parents
    parents: list                  # depth-(l-1) box cut by each separator (same order)


@dataclass
class NestedDissection:
    nx: int
    ny: int
    leaf: int
    L: int
    perm: np.ndarray               # perm[i] = grid node of the i-th unknown in order I
    leaves: list                   # depth-L boxes, depth-first order
    seps: dict                     # level -> list of (parent box, node array)
    levels: dict = field(default_factory=dict)   # level -> Level

    @property
    def N(self):
        return self.nx * self.ny


def _cut(box: Box):
    """Straight middle separator of a box and its two children (Alg. 1 lines 5-9)."""
    if box.w < box.h:   # separating direction along x: a horizontal line
        ym = box.y0 + (box.h - 1) // 2
        nodes = [(x, ym) for x in range(box.x0, box.x1 + 1)]
        c1 = Box(box.x0, box.x1, box.y0, ym - 1, box.depth + 1)
        c2 = Box(box.x0, box.x1, ym + 1, box.y1, box.depth + 1)
        return "H", nodes, c1, c2
    xm = box.x0 + (box.w - 1) // 2
    nodes = [(xm, y) for y in range(box.y0, box.y1 + 1)]
    c1 = Box(box.x0, xm - 1, box.y0, box.y1, box.depth + 1)
    c2 = Box(xm + 1, box.x1, box.y0, box.y1, box.depth + 1)
    return "V", nodes, c1, c2


def _valid(n: int, leaf: int) -> bool:
    q, r = divmod(n + 1, leaf + 1)
    return r == 0 and q >= 1 and (q & (q - 1)) == 0


def nested_dissection(nx: int, ny: int, leaf: int = 15) -> NestedDissection:
    """Alg. 1 specialised to a regular nx x ny grid (natural node id x + nx*y)."""
    if not (_valid(nx, leaf) and _valid(ny, leaf)):
        raise ValueError("grid sides must be (leaf+1)*2^k - 1")
    L = int(round(math.log2((nx + 1) // (leaf + 1)))) + int(round(math.log2((ny + 1) // (leaf + 1))))
    leaves: list = []
    seps: dict = {l: [] for l in range(1, L + 1)}
    boxes_at: dict = {d: [] for d in range(0, L + 1)}

    def rec(box: Box, l: int):
        boxes_at[box.depth].append(box)
        if box.w == leaf and box.h == leaf:
            leaves.append(box)
            return
        _, nodes, c1, c2 = _cut(box)
        seps[l].append((box, np.array([x + nx * y for x, y in nodes], dtype=np.int64)))
        rec(c1, l + 1)
        rec(c2, l + 1)

    rec(Box(0, nx - 1, 0, ny - 1, 0), 1)
    order = []
    for b in leaves:
        for y in range(b.y0, b.y1 + 1):
            for x in range(b.x0, b.x1 + 1):
                order.append(x + nx * y)
    for l in range(L, 0, -1):
        for _, nodes in seps[l]:
            order.extend(nodes.tolist())
    nd = NestedDissection(nx, ny, leaf, L, np.array(order, dtype=np.int64), leaves, seps)
    for l in range(1, L + 1):
        nd.levels[l] = _level(nd, l, boxes_at[l])
    return nd


def _sides(box: Box, nx: int, ny: int):
    """Keys and node lists of the existing sides of a box (bottom, top, left, right)."""
    out = []
    if box.y0 > 0:
        y = box.y0 - 1
        out.append((("H", y, box.x0, box.x1), [x + nx * y for x in range(box.x0, box.x1 + 1)]))
    if box.y1 < ny - 1:
        y = box.y1 + 1
        out.append((("H", y, box.x0, box.x1), [x + nx * y for x in range(box.x0, box.x1 + 1)]))
    if box.x0 > 0:
        x = box.x0 - 1
        out.append((("V", x, box.y0, box.y1), [x + nx * y for y in range(box.y0, box.y1 + 1)]))
    if box.x1 < nx - 1:
        x = box.x1 + 1
        out.append((("V", x, box.y0, box.y1), [x + nx * y for y in range(box.y0, box.y1 + 1)]))
    return out


def box_corners(box: Box, nx: int, ny: int):
    """Grid nodes of the existing corners of a box (crossings not on the boundary)."""
    out = []
    for x in (box.x0 - 1, box.x1 + 1):
        for y in (box.y0 - 1, box.y1 + 1):
            if 0 <= x < nx and 0 <= y < ny:
                out.append(x + nx * y)
    return sorted(out)


def segment_id(key, w: int, h: int, nx: int, ny: int) -> int:
    """Index of a level segment in the tiling of depth-l boxes (w x h each): horizontal
    sides first (by box column, then line), then vertical sides.  Used to key the sketch."""
    bx, by = (nx + 1) // (w + 1), (ny + 1) // (h + 1)
    if key[0] == "H":
        I = key[2] // (w + 1)
        J = (key[1] + 1) // (h + 1)
        return I + bx * (J - 1)
    I = (key[1] + 1) // (w + 1)
    J = key[2] // (h + 1)
    return bx * (by - 1) + (I - 1) + (bx - 1) * J


def _level(nd: NestedDissection, l: int, boxes: list) -> Level:
    segs: dict = {}
    corners = set()
    w, h = boxes[0].w, boxes[0].h
    sep_keys = set()
    parents, sep_list = [], []
    for parent, nodes in nd.seps[l]:
        kind, _, c1, _ = _cut(parent)
        if kind == "H":
            key = ("H", c1.y1 + 1, parent.x0, parent.x1)
        else:
            key = ("V", c1.x1 + 1, parent.y0, parent.y1)
        sep_keys.add(key)
        sep_list.append(key)
        parents.append(parent)
    for b in boxes:
        for key, nodes in _sides(b, nd.nx, nd.ny):
            if key not in segs:
                segs[key] = Segment(key, l, segment_id(key, w, h, nd.nx, nd.ny),
                                    np.array(nodes, dtype=np.int64), [], key in sep_keys)
            segs[key].boxes.append(b)
        corners.update(box_corners(b, nd.nx, nd.ny))
    return Level(l, boxes, segs, sorted(corners), sep_list, parents)


def chebyshev_to_segment(key, node: int, nx: int) -> int:
    """Chebyshev grid distance from a node to the geometric extent of a segment."""
    x, y = node % nx, node // nx
    if key[0] == "H":
        return max(abs(y - key[1]), max(0, key[2] - x, x - key[3]))
    return max(abs(x - key[1]), max(0, key[2] - y, y - key[3]))


def separator_walk(coords: np.ndarray, adj: list, boundary=None, theta: float = 0.1) -> list:
    """Literal restatement of the separator search of Sec. 3.1 on a general graph.

    coords: (n, 2) vertex coordinates; adj: neighbour lists; boundary: boolean mask of the
    vertices on the boundary of the subgraph (default: vertices with fewer neighbours than
    the most connected one).  The centre vertex is the vertex closest to the coordinate
    median; the separating direction d is +x when the bounding box is narrower than tall,
    else +y; the walk repeatedly moves to the neighbour maximising D(u, v, c, d) of
    Eq. (degreebias) while D > 0, first along +d, then along -d.

    Reading: Sec. 3.1 stops a walk when the next vertex is missing or D <= 0; on a grid the
    second term of D stays positive along the subgraph's edge, so the walk here also ends
    at the first boundary vertex it reaches (the separator has then cut the subgraph).
    Returns the separator as a list of vertex indices from the -d end to the +d end.
    """
    if boundary is None:
        deg = np.array([len(a) for a in adj])
        boundary = deg < deg.max()
    med = np.median(coords, axis=0)
    d2 = np.sum((coords - med) ** 2, axis=1)
    c = int(np.argmin(d2))   # ties -> lowest index
    width = coords[:, 0].max() - coords[:, 0].min()
    height = coords[:, 1].max() - coords[:, 1].min()
    d = np.array([1.0, 0.0]) if width < height else np.array([0.0, 1.0])

    def D(u, v, dd):
        a = coords[u] - coords[v]
        b = coords[u] - coords[c]
        t1 = float(a @ dd) / (np.linalg.norm(a) * np.linalg.norm(dd))
        nb = np.linalg.norm(b)
        t2 = 0.0 if nb == 0 else float(b @ dd) / (nb * np.linalg.norm(dd))
        return t1 + theta * t2

    def walk(dd):
        path, v, seen = [], c, {c}
        while True:
            best, bestu = None, None
            for u in adj[v]:
                if u in seen:
                    continue
                val = D(u, v, dd)
                if best is None or val > best:
                    best, bestu = val, u
            if bestu is None or best <= 0:
                return path
            path.append(bestu)
            seen.add(bestu)
            if boundary[bestu]:
                return path
            v = bestu

    fwd = walk(d)
    bwd = walk(-d)
    return bwd[::-1] + [c] + fwd
