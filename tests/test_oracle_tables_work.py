"""Pins of the oracle's per-level index tables and of its algorithmic work counts (no GPU).

The tables: at eps_ID = 0 nothing is truncated and the merge E_(l) concatenates whole
children (Sec. 4.3), so every segment of every level holds exactly the grid nodes of its box
side in increasing coordinate, which the geometry alone fixes; at eps_ID > 0 each merged
segment is the skeleton of its first child, the junction, then the skeleton of its second
child.  The work counts (oracle/flops.py, the cost terms of Sec. 5.2) are pinned by closed
forms and by brute-force operation counting on small blocks.
"""
import numpy as np
import pytest

import workloads as W
from oracle import flops as fl
from oracle.nd import nested_dissection
from oracle.spalu import Options, factor


def _geometric_nodes(key, nx):
    """Grid nodes of a box side from its key alone: ('H', y, x0, x1) or ('V', x, y0, y1)."""
    if key[0] == "H":
        return np.array([x + nx * key[1] for x in range(key[2], key[3] + 1)])
    return np.array([key[1] + nx * y for y in range(key[2], key[3] + 1)])


@pytest.mark.parametrize("nx,ny", [(63, 63), (127, 31), (31, 63)])
def test_eps0_level_tables_are_the_geometry(nx, ny):
    P = W.make_problem("diffusion", nx, seed=5, nrhs=1, ny=ny)
    nd = nested_dissection(nx, ny)
    F = factor(P.A, nd, Options(eps=0.0, symmetric=True))
    for l in range(1, nd.L + 1):
        st = F.stats["levels"][l]
        segs = nd.levels[l].segments
        assert sorted(st["nodes"]) == sorted(s.sid for s in segs.values())
        for key, seg in segs.items():
            geo = _geometric_nodes(key, nx)
            assert np.array_equal(st["nodes"][seg.sid], geo)
            assert np.array_equal(st["skel"][seg.sid], geo)          # k = e, identity order


def test_merged_segments_concatenate_child_skeletons():
    """eps > 0: a level-(l-1) segment split at level l is [skeleton of the lower/left piece,
    junction, skeleton of the upper/right piece]; an unsplit side is the skeleton of its one
    piece."""
    n = 127
    P = W.make_problem("diffusion", n, seed=6, nrhs=1)
    nd = nested_dissection(n, n)
    F = factor(P.A, nd, Options(eps=1e-6, symmetric=True))
    for l in range(nd.L, 1, -1):
        fine, coarse = nd.levels[l], nd.levels[l - 1]
        st, up = F.stats["levels"][l], F.stats["levels"][l - 1]
        kk = dict(zip(sorted(s.sid for s in fine.segments.values()), st["ranks"]))
        for key, seg in coarse.segments.items():
            pieces = [s for k2, s in fine.segments.items()
                      if k2[0] == key[0] and k2[1] == key[1] and key[2] <= k2[2] and k2[3] <= key[3]]
            pieces.sort(key=lambda s: s.key[2])
            expect = []
            for i, s in enumerate(pieces):
                if i:
                    a = pieces[i - 1].key[3] + 1                        # the junction between
                    expect.append(a + n * key[1] if key[0] == "H" else key[1] + n * a)
                expect.extend(st["skel"][s.sid][:kk[s.sid]].tolist())
            assert up["nodes"][seg.sid].tolist() == expect


def test_lu_count_closed_form_and_brute_force():
    for n in range(0, 40):
        assert fl.lu(n) == n * (n - 1) * (4 * n + 1) // 6
    # brute force: count the divisions, multiplications and subtractions of a literal GEPP
    for n in (1, 2, 5, 9):
        ops = 0
        for j in range(n):
            for i in range(j + 1, n):
                ops += 1                                   # multiplier
                for c in range(j + 1, n):
                    ops += 2                               # a_ic -= l_ij u_jc
        assert fl.lu(n) == ops


def test_qr_count_brute_force():
    """Operations of a literal Householder step loop: norm of the column below the diagonal,
    then for each trailing column a dot product and an update."""
    for m, e, k in [(7, 5, 3), (20, 9, 9), (4, 6, 4), (3, 8, 5), (10, 1, 1)]:
        ops = 0
        for j in range(min(k, m, e)):
            ops += 2 * (m - j)                             # sum of squares
            for c in range(j + 1, e):
                ops += 2 * (m - j) + 2 * (m - j)           # v . y, then y -= tau v (v . y)
        assert fl.qr(m, e, k) == ops
    assert fl.sketch(3, 4, 5) == 2 * 3 * 4 * 5
    assert fl.interp(4, 9) == 4 * 4 * 5 and fl.interp(0, 9) == 0
    assert fl.apply(10, 10) == 0 and fl.apply(10, 0) == 0 and fl.apply(10, 4) == 4 * 10 * 4 * 6
    assert fl.elim(3, 0) == fl.lu(3) and fl.elim(3, 2) == fl.lu(3) + 2 * 9 * 2 + 2 * 4 * 3


@pytest.mark.parametrize("nx,ny", [(63, 63), (127, 31)])
def test_eps0_work_counts_closed_form(nx, ny):
    """eps = 0: no ID is computed (sparsify count 0) and every level-l separator, whole, is
    eliminated against every unknown on its parent box's boundary: the full lengths of the
    parent's sides that lie inside the grid plus its corners that lie inside."""
    P = W.make_problem("diffusion", nx, seed=7, nrhs=1, ny=ny)
    nd = nested_dissection(nx, ny)
    F = factor(P.A, nd, Options(eps=0.0, symmetric=True))
    for l in range(1, nd.L + 1):
        want = 0
        for (parent, sep) in nd.seps[l]:
            w, h = parent.x1 - parent.x0 + 1, parent.y1 - parent.y0 + 1
            inside_x = [parent.x0 > 0, parent.x1 < nx - 1]
            inside_y = [parent.y0 > 0, parent.y1 < ny - 1]
            dP = w * sum(inside_y) + h * sum(inside_x) + sum(a and b for a in inside_x for b in inside_y)
            want += fl.elim(sep.size, dP)
        assert F.stats["levels"][l]["flops_merge"] == want
        assert F.stats["levels"][l]["flops_sparsify"] == 0


def test_work_counts_grow_linearly_with_n():
    """Sec. 5.2: with bounded ranks the factorization work tends to O(N): the work per unknown
    grows ever more slowly as the grid is refined (coarse segments reach their rank bound)."""
    per = []
    for n in (63, 127, 255):
        P = W.make_problem("diffusion", n, seed=8, nrhs=1)
        F = factor(P.A, nested_dissection(n, n), Options(eps=1e-6, symmetric=True))
        tot = sum(v["flops_sparsify"] + v["flops_merge"] for v in F.stats["levels"].values())
        per.append(tot / (n * n))
    r1, r2 = per[1] / per[0], per[2] / per[1]
    assert r2 < 1.5 and r2 < r1, per
