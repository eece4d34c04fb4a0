"""Algorithmic work counts of the method (floating-point operations, one multiply-add = 2).

Test infrastructure: the oracle's factorization adds these counts up per level, and the
benchmark divides the same counts (accumulated by the CUDA kernels with the same formulas) by
the measured kernel times.  They follow the cost terms of Sec. 5.2 ("Complexity of
factorization based on low rank approximations"): the sampled interaction block, the
column-pivoted QR behind each ID, the interpolation matrix, the sparsifying transforms and the
block eliminations; the paper gives their orders, the exact sums below are this project's
definitions, written for the operations the method itself needs (no padding, no avoided
dense work).

  lu(n)            LU with partial pivoting of an n x n block: at step j, n-j-1 divisions and
                   an (n-j-1) x (n-j-1) rank-one update.
  sketch(h, f, e)  G (h x f) times B_F (f x e).
  qr(m, e, k)      k Householder steps on an m x e block: reflector norm (2 (m-j)) and its
                   application to the e-j-1 trailing columns (4 (m-j)(e-j-1)).
  interp(k, e)     T = R_11^{-1} R_12: e-k back substitutions of order k.
  apply(e, k)      the column and row operations of Eq. (UtALt) on the segment's own e x e
                   block: 2 e k (e-k) each.
  elim(p, q)       elimination of p unknowns against q neighbours (Eq. (L^-1 A U^-1)):
                   lu(p), W = L^{-1} P A_pq and Z = A_qp U^{-1} (p^2 q each), and the Schur
                   update A_qq -= Z W (2 q^2 p).
"""
from __future__ import annotations


def lu(n: int) -> int:
    return sum((n - j - 1) + 2 * (n - j - 1) ** 2 for j in range(n))


def sketch(h: int, f: int, e: int) -> int:
    return 2 * h * f * e


def qr(m: int, e: int, k: int) -> int:
    return sum(2 * (m - j) + 4 * (m - j) * (e - j - 1) for j in range(min(k, m, e)))


def interp(k: int, e: int) -> int:
    return k * k * (e - k)


def apply(e: int, k: int) -> int:
    return 4 * e * k * (e - k)


def elim(p: int, q: int) -> int:
    return lu(p) + 2 * p * p * q + 2 * q * q * p
