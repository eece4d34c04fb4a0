"""Seeded synthetic workloads: 5-point finite-difference matrices on regular grids and RHS.

This module defines the *problems* the solver is run on; it holds none of the solver's
arithmetic.  Both the CPU oracle (``oracle/``) and the CUDA path consume its output, and
nothing here imports either of them.

Grid convention (shared by every consumer):
  * ``nx`` x ``ny`` interior nodes of the unit square, spacing ``hx = 1/(nx+1)``,
    ``hy = 1/(ny+1)``; node ``(i, j)`` sits at ``((i+1) hx, (j+1) hy)``.
  * natural index ``g = i + nx * j`` (x fastest).
  * Dirichlet ``u = 0`` on the boundary; boundary nodes are eliminated, so the matrix is
    ``N x N`` with ``N = nx * ny``.
  * CSR with int32 ``indptr``/``indices`` (columns sorted within a row) and float64 data.

The paper's experiments use FEM meshes and random fields that are not available
(Sec. 6); these finite-difference analogues stand in for them:
  * ``laplace``     : -Lap_h u = f                          (symmetric positive definite)
  * ``diffusion``   : -div(a grad u) = f, a = exp(GRF)       (symmetric positive definite)
  * ``helmholtz``   : -Lap_h u - k^2(x) u = f                (symmetric indefinite)
  * ``convdiff``    : -Lap_h u + beta . grad u = f, upwind   (non-symmetric)
  * ``aniso``       : -d/dx(a1 du/dx) - d/dy(a2 du/dy) + beta . grad u = f, a1 = exp(GRF),
                      a2 = 10 exp(GRF') (a diagonal anisotropic coefficient, a tenfold
                      contrast between the directions), first-order upwind convection
                      (non-symmetric; the 5-point analogue of Sec. 6.4's problem)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CSR", "Problem", "laplace", "diffusion", "helmholtz", "convdiff", "grf",
    "rhs_normal", "rhs_point_sources", "make_problem", "grid_sizes_ok", "predictor_init_params",
    "aniso",
]


@dataclass
class CSR:
    n: int
    indptr: np.ndarray   # int32 [n+1]
    indices: np.ndarray  # int32 [nnz]
    data: np.ndarray     # float64 [nnz]

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        for r in range(self.n):
            s, e = self.indptr[r], self.indptr[r + 1]
            a[r, self.indices[s:e]] += self.data[s:e]
        return a

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """y = A x for x of shape (n,) or (n, k) (row-by-row gather; used by tests)."""
        rows = np.repeat(np.arange(self.n), np.diff(self.indptr))
        contrib = self.data[:, None] * np.asarray(x).reshape(self.n, -1)[self.indices]
        y = np.zeros((self.n, contrib.shape[1]))
        np.add.at(y, rows, contrib)
        return y.reshape(np.asarray(x).shape)


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    A: CSR
    B: np.ndarray                    # (N, nrhs), column-major when copied to the device
    symmetric: bool
    meta: dict = field(default_factory=dict)


def grid_sizes_ok(nx: int, ny: int, leaf: int = 15) -> bool:
    """True when both sides are leaf+1 times a power of two, minus one (e.g. 15, 31, ..., 1023)."""
    def ok(n):
        q, r = divmod(n + 1, leaf + 1)
        return r == 0 and q >= 1 and (q & (q - 1)) == 0
    return ok(nx) and ok(ny)


def _assemble(nx: int, ny: int, diag: np.ndarray, west, east, south, north) -> CSR:
    """Build CSR from per-node stencil weights (arrays of shape (ny, nx)).

    Off-diagonal weights that point at a boundary node are dropped (Dirichlet u=0).
    """
    n = nx * ny
    rows, cols, vals = [], [], []
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    g = ii + nx * jj
    entries = [
        (diag, 0, 0),
        (west, -1, 0),
        (east, 1, 0),
        (south, 0, -1),
        (north, 0, 1),
    ]
    for w, di, dj in entries:
        i2, j2 = ii + di, jj + dj
        m = (i2 >= 0) & (i2 < nx) & (j2 >= 0) & (j2 < ny)
        rows.append(g[m])
        cols.append((i2 + nx * j2)[m])
        vals.append(np.broadcast_to(w, (ny, nx))[m])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals).astype(np.float64)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(indptr, r + 1, 1)
    indptr = np.cumsum(indptr)
    return CSR(n, indptr.astype(np.int32), c.astype(np.int32), v)


def laplace(nx: int, ny: int) -> CSR:
    """Standard 5-point -Lap_h with Dirichlet boundary (h^-2 scaled)."""
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    ax, ay = 1.0 / hx**2, 1.0 / hy**2
    shape = (ny, nx)
    return _assemble(nx, ny, np.full(shape, 2 * ax + 2 * ay), np.full(shape, -ax),
                     np.full(shape, -ax), np.full(shape, -ay), np.full(shape, -ay))


def diffusion(nx: int, ny: int, a_nodes: np.ndarray) -> CSR:
    """-div(a grad u) with a sampled on the (ny+2) x (nx+2) node lattice (boundary ring
    included); the face coefficient is the arithmetic mean of its two nodal values."""
    assert a_nodes.shape == (ny + 2, nx + 2)
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    P = a_nodes[1:-1, 1:-1]
    aw = 0.5 * (P + a_nodes[1:-1, :-2]) / hx**2
    ae = 0.5 * (P + a_nodes[1:-1, 2:]) / hx**2
    as_ = 0.5 * (P + a_nodes[:-2, 1:-1]) / hy**2
    an = 0.5 * (P + a_nodes[2:, 1:-1]) / hy**2
    return _assemble(nx, ny, aw + ae + as_ + an, -aw, -ae, -as_, -an)


def helmholtz(nx: int, ny: int, k2_interior: np.ndarray) -> CSR:
    """-Lap_h - diag(k^2) with k^2 given at the interior nodes, shape (ny, nx)."""
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    ax, ay = 1.0 / hx**2, 1.0 / hy**2
    shape = (ny, nx)
    return _assemble(nx, ny, 2 * ax + 2 * ay - k2_interior, np.full(shape, -ax),
                     np.full(shape, -ax), np.full(shape, -ay), np.full(shape, -ay))


def aniso(nx: int, ny: int, a1_nodes: np.ndarray, a2_nodes: np.ndarray, beta: tuple[float, float]) -> CSR:
    """-d/dx(a1 du/dx) - d/dy(a2 du/dy) + beta . grad u with a1, a2 on the (ny+2) x (nx+2) node
    lattice (x faces take the mean of a1 over their two nodes, y faces the mean of a2) and
    first-order upwind convection (non-symmetric)."""
    assert a1_nodes.shape == (ny + 2, nx + 2) and a2_nodes.shape == (ny + 2, nx + 2)
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    P1, P2 = a1_nodes[1:-1, 1:-1], a2_nodes[1:-1, 1:-1]
    w = -0.5 * (P1 + a1_nodes[1:-1, :-2]) / hx**2
    e = -0.5 * (P1 + a1_nodes[1:-1, 2:]) / hx**2
    s_ = -0.5 * (P2 + a2_nodes[:-2, 1:-1]) / hy**2
    n = -0.5 * (P2 + a2_nodes[2:, 1:-1]) / hy**2
    d = -(w + e + s_ + n)
    bx, by = beta
    if bx > 0:
        d, w = d + bx / hx, w - bx / hx
    else:
        d, e = d - bx / hx, e + bx / hx
    if by > 0:
        d, s_ = d + by / hy, s_ - by / hy
    else:
        d, n = d - by / hy, n + by / hy
    return _assemble(nx, ny, d, w, e, s_, n)


def convdiff(nx: int, ny: int, beta: tuple[float, float]) -> CSR:
    """-Lap_h u + beta . grad u with first-order upwind differences (non-symmetric)."""
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    bx, by = beta
    shape = (ny, nx)
    d = np.full(shape, 2 / hx**2 + 2 / hy**2)
    w = np.full(shape, -1 / hx**2)
    e = np.full(shape, -1 / hx**2)
    s = np.full(shape, -1 / hy**2)
    n = np.full(shape, -1 / hy**2)
    if bx > 0:      # bx (u_P - u_W) / hx
        d = d + bx / hx
        w = w - bx / hx
    else:           # bx (u_E - u_P) / hx
        d = d - bx / hx
        e = e + bx / hx
    if by > 0:
        d = d + by / hy
        s = s - by / hy
    else:
        d = d - by / hy
        n = n + by / hy
    return _assemble(nx, ny, d, w, e, s, n)


def grf(nx: int, ny: int, ell: float, var: float, rng: np.random.Generator) -> np.ndarray:
    """Zero-mean Gaussian random field with covariance var*exp(-r^2/(2 ell^2)) on the
    (ny+2) x (nx+2) node lattice (boundary ring included), by circulant embedding on a
    periodic grid at least twice the lattice (Dietrich & Newsam 1997).  Eigenvalues of the
    embedding below 1e-10 of the largest are set to zero: the squared-exponential spectrum
    decays so fast that most of them are FFT rounding noise (either sign, ~1e-16 of the
    largest), whose square roots would otherwise add platform-dependent amplitudes of ~1e-8
    to the field; what is dropped carries less than 1e-10 of the variance."""
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    mx = 1 << int(math.ceil(math.log2(2 * (nx + 2))))
    my = 1 << int(math.ceil(math.log2(2 * (ny + 2))))
    dx = np.minimum(np.arange(mx), mx - np.arange(mx)) * hx
    dy = np.minimum(np.arange(my), my - np.arange(my)) * hy
    c = var * np.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (2 * ell**2))
    lam = np.fft.fft2(c).real
    lam = np.where(lam > 1e-10 * lam.max(), lam, 0.0)
    z = rng.standard_normal((my, mx)) + 1j * rng.standard_normal((my, mx))
    f = np.fft.fft2(np.sqrt(lam / (mx * my)) * z)
    return np.ascontiguousarray(f.real[: ny + 2, : nx + 2])


def rhs_normal(n: int, nrhs: int, rng: np.random.Generator) -> np.ndarray:
    return rng.standard_normal((n, nrhs))


def rhs_point_sources(nx: int, ny: int, nrhs: int, rng: np.random.Generator) -> np.ndarray:
    """Gaussian bumps exp(-|x-c|^2 / (2 (2h)^2)) with centres c ~ U[0.1, 0.9]^2."""
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    h = max(hx, hy)
    xs = (np.arange(nx) + 1) * hx
    ys = (np.arange(ny) + 1) * hy
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    out = np.empty((nx * ny, nrhs))
    for k in range(nrhs):
        cx, cy = rng.uniform(0.1, 0.9, size=2)
        out[:, k] = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * (2 * h) ** 2)).ravel()
    return out


def make_problem(kind: str, n: int, seed: int = 0, nrhs: int | None = None,
                 ny: int | None = None) -> Problem:
    """Build one of the synthetic problem families on an n x ny grid (ny defaults to n).

    kind: 'laplace' (1 RHS), 'diffusion' (16 RHS, a=exp(GRF, ell=0.05, var=1)),
          'helmholtz' (8 point-source RHS, 10 points per wavelength, k^2 perturbed by 20%
          of a GRF rescaled to max|s|=1), 'convdiff' (4 RHS, beta=50(cos t, sin t), t~U[0,2pi)).
    """
    nyy = n if ny is None else ny
    rng = np.random.default_rng(seed)
    N = n * nyy
    if kind == "laplace":
        A = laplace(n, nyy)
        B = rhs_normal(N, nrhs or 1, rng)
        return Problem(kind, n, nyy, A, B, True, {})
    if kind == "diffusion":
        g = grf(n, nyy, 0.05, 1.0, rng)
        A = diffusion(n, nyy, np.exp(g))
        B = rhs_normal(N, nrhs or 16, rng)
        return Problem(kind, n, nyy, A, B, True, {"ell": 0.05, "var": 1.0})
    if kind == "helmholtz":
        h = 1.0 / (max(n, nyy) + 1)
        k0 = 2 * math.pi / (10 * h)
        s = grf(n, nyy, 0.05, 1.0, rng)[1:-1, 1:-1]
        s = s / np.max(np.abs(s))
        k2 = k0**2 * (1 + 0.2 * s)
        A = helmholtz(n, nyy, k2)
        B = rhs_point_sources(n, nyy, nrhs or 8, rng)
        return Problem(kind, n, nyy, A, B, True, {"k0": k0})
    if kind == "convdiff":
        theta = rng.uniform(0, 2 * math.pi)
        beta = (50 * math.cos(theta), 50 * math.sin(theta))
        A = convdiff(n, nyy, beta)
        B = rhs_normal(N, nrhs or 4, rng)
        return Problem(kind, n, nyy, A, B, False, {"beta": beta})
    if kind == "aniso":
        g1 = grf(n, nyy, 0.05, 1.0, rng)
        g2 = grf(n, nyy, 0.05, 1.0, rng)
        theta = rng.uniform(0, 2 * math.pi)
        beta = (50 * math.cos(theta), 50 * math.sin(theta))
        A = aniso(n, nyy, np.exp(g1), 10.0 * np.exp(g2), beta)
        B = rhs_normal(N, nrhs or 4, rng)
        return Problem(kind, n, nyy, A, B, False, {"beta": beta, "ratio": 10.0})
    raise ValueError(f"unknown problem kind {kind!r}")


def predictor_init_params(seed: int, nfeat: int = 16, nhid: int = 64, nout: int = 2) -> np.ndarray:
    """Seeded initial weights of the rank predictor's 16 -> 64 -> 2 network (float32):
    He-normal W1 (nhid x nfeat, row-major) and W2 (nout x nhid), zero biases, packed as
    W1 | b1 | W2 | b2 (the parameter layout of the library's predictor entry points).  A
    seeded draw, like the right-hand sides: an input to both the oracle and the device."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((nhid, nfeat)) * math.sqrt(2.0 / nfeat)
    W2 = rng.standard_normal((nout, nhid)) * math.sqrt(2.0 / nhid)
    return np.concatenate([W1.ravel(), np.zeros(nhid), W2.ravel(), np.zeros(nout)]).astype(np.float32)
