"""Nested dissection of a general graph with coordinates (Sec. 3.1, Alg. 1): the oracle and
the library's host implementation (`spalu_nd_order_csr`).  No GPU.

The oracle is pinned by the special case the paper's construction reduces to: on a regular
grid (leaf size 225) the walk gives the straight middle cuts, so the ordering must equal the
grid dissection's order I bit for bit, on square and rectangular grids; and on irregular
meshes by invariants: the order is a permutation, every separator cuts its part (no edge
joins two different leaves), separators shrink level by level.  The library must equal the
oracle bit for bit on grids, jittered grids and Delaunay meshes of random points.
"""
import numpy as np
import pytest

import workloads as W
from oracle.nd import nested_dissection
from oracle.nd_graph import nested_dissection_graph


@pytest.fixture(scope="module")
def lib():
    from paper_2408_14193_gb300 import build, load_library
    build.build()
    return load_library()


def _grid(nx, ny, jitter=0.0, seed=0):
    A = W.laplace(nx, ny)
    xs, ys = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    xy = np.stack([xs.ravel(), ys.ravel()], 1).astype(float)
    if jitter:
        xy += np.random.default_rng(seed).uniform(-jitter, jitter, xy.shape)
    return A.indptr, A.indices, xy


def _delaunay(npts, seed):
    sp = pytest.importorskip("scipy.spatial")
    pts = np.random.default_rng(seed).random((npts, 2))
    tri = sp.Delaunay(pts)
    ip, ix = tri.vertex_neighbor_vertices
    bd = np.zeros(npts, dtype=bool)
    bd[np.unique(tri.convex_hull)] = True
    return ip, ix, pts, bd


def _leaves_separated(ip, ix, perm, level):
    """Every edge between two non-separator vertices stays inside one component of the graph
    without its separators, and no component is larger than its share."""
    n = len(perm)
    sep = level > 0
    comp = -np.ones(n, dtype=np.int64)
    k = 0
    for v in range(n):
        if sep[v] or comp[v] >= 0:
            continue
        comp[v] = k
        stack = [v]
        while stack:
            x = stack.pop()
            for u in ix[ip[x]:ip[x + 1]]:
                if not sep[u] and comp[u] < 0:
                    comp[u] = k
                    stack.append(u)
        k += 1
    # the leaves in order I are contiguous runs of one component each
    nleaf_vertices = int((~sep).sum())
    runs = comp[perm[:nleaf_vertices]]
    changes = np.count_nonzero(np.diff(runs)) + 1
    return k, changes


@pytest.mark.parametrize("nx,ny", [(15, 15), (31, 31), (63, 63), (127, 31), (31, 127), (255, 63)])
def test_oracle_graph_dissection_is_the_grid_dissection(nx, ny):
    ip, ix, xy = _grid(nx, ny)
    perm, level = nested_dissection_graph(xy, ip, ix, 225)
    nd = nested_dissection(nx, ny)
    assert np.array_equal(perm, nd.perm)
    assert level.max() == nd.L
    for l in range(1, nd.L + 1):                  # separator vertices of each level
        want = np.sort(np.concatenate([s for _, s in nd.seps[l]]))
        assert np.array_equal(np.sort(np.nonzero(level == l)[0]), want)


@pytest.mark.parametrize("case", ["jitter", "delaunay"])
def test_oracle_graph_dissection_invariants(case):
    if case == "jitter":
        ip, ix, xy = _grid(63, 63, jitter=0.3, seed=1)
        bd = None
        leaf = 100
    else:
        ip, ix, xy, bd = _delaunay(3000, 2)
        leaf = 64
    perm, level = nested_dissection_graph(xy, ip, ix, leaf, bd)
    n = xy.shape[0]
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert level.max() >= 4
    k, changes = _leaves_separated(ip, ix, perm, level)
    assert changes == k                             # every component one contiguous run of leaves
    sizes = [int((level == l).sum()) for l in range(1, level.max() + 1)]
    assert sizes[0] >= 1 and all(s > 0 for s in sizes)


@pytest.mark.parametrize("nx,ny", [(63, 63), (127, 31), (255, 255)])
def test_library_equals_grid_dissection(lib, nx, ny):
    from paper_2408_14193_gb300.spalu import nd_order_csr
    ip, ix, xy = _grid(nx, ny)
    perm, level = nd_order_csr(ip, ix, xy, 225)
    assert np.array_equal(perm.astype(np.int64), nested_dissection(nx, ny).perm)


@pytest.mark.parametrize("case,leaf", [("jitter", 100), ("delaunay3000", 64), ("delaunay20000", 100)])
def test_library_equals_oracle_bit_exact(lib, case, leaf):
    from paper_2408_14193_gb300.spalu import nd_order_csr
    if case == "jitter":
        ip, ix, xy = _grid(127, 63, jitter=0.3, seed=3)
        bd = None
    else:
        ip, ix, xy, bd = _delaunay(int(case[8:]), 4)
    po, lo = nested_dissection_graph(xy, ip, ix, leaf, bd)
    pc, lc = nd_order_csr(ip, ix, xy, leaf, bd)
    assert np.array_equal(po, pc.astype(np.int64))
    assert np.array_equal(lo, lc.astype(np.int64))


def test_library_rejects_bad_arguments(lib):
    import ctypes
    from paper_2408_14193_gb300.spalu import SpaluError, nd_order_csr
    ip, ix, xy = _grid(15, 15)
    bad = ix.copy()
    bad[3] = 10_000
    with pytest.raises(SpaluError):
        nd_order_csr(ip, bad, xy, 16)
    xyn = xy.copy()
    xyn[5, 0] = np.nan
    with pytest.raises(SpaluError):
        nd_order_csr(ip, ix, xyn, 16)
    assert lib.spalu_nd_order_csr(4, None, None, None, None, 8, None, None) == -1
