"""Dense building blocks of the oracle, in plain FP64 loops.

  gepp / lu_solve  - Gaussian elimination with partial pivoting (pivot = largest |entry| in
                     the column, ties -> lowest row), used for every "straightforward LU"
                     of Sec. 4.3 (leaf interiors, remainders, separators).
  cpqr             - Householder QR with column pivoting (Businger-Golub), the permutation
                     Pi of Eq. (RRQR 1); column norms are downdated and recomputed when the
                     downdate loses accuracy (Drmac & Bujanovic, 2008).
  interp_decomp    - the interpolative decomposition of Eq. (RRQR 2): k skeleton columns
                     and T = R_1^{-1} R_2, truncated at the first |R_kk| <= eps |R_11|.
"""
from __future__ import annotations

import numpy as np

TIE_RTOL = 1e-12     # column norms within this relative distance of the largest are ties
TOL3Z = float(np.sqrt(np.finfo(np.float64).eps))


class SingularPivot(ArithmeticError):
    pass


def gepp(A: np.ndarray):
    """LU with partial pivoting: returns (lu, piv) with P A = L U, L unit lower (stored
    below the diagonal), piv[j] = row exchanged with row j at step j."""
    a = np.array(A, dtype=np.float64, copy=True)
    n = a.shape[0]
    piv = np.arange(n)
    for j in range(n):
        p = j + int(np.argmax(np.abs(a[j:, j])))     # first maximum: ties -> lowest row
        if a[p, j] == 0.0:
            raise SingularPivot(f"zero pivot at column {j}")
        if p != j:
            a[[j, p], :] = a[[p, j], :]
            piv[j] = p
        a[j + 1:, j] /= a[j, j]
        a[j + 1:, j + 1:] -= np.outer(a[j + 1:, j], a[j, j + 1:])
    return a, piv


def lu_solve(lu: np.ndarray, piv: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve A x = b from gepp's output; b may have several columns."""
    x = np.array(b, dtype=np.float64, copy=True)
    n = lu.shape[0]
    for j in range(n):
        if piv[j] != j:
            x[[j, piv[j]]] = x[[piv[j], j]]
    for j in range(n):                       # unit lower triangular
        x[j + 1:] -= np.multiply.outer(lu[j + 1:, j], x[j])
    for j in range(n - 1, -1, -1):           # upper triangular
        x[j] = x[j] / lu[j, j]
        x[:j] -= np.multiply.outer(lu[:j, j], x[j])
    return x


def solve_upper(R: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Back substitution R X = B for upper-triangular R."""
    X = np.array(B, dtype=np.float64, copy=True)
    k = R.shape[0]
    for i in range(k - 1, -1, -1):
        X[i] = (X[i] - R[i, i + 1:] @ X[i + 1:]) / R[i, i]
    return X


def _pivot(vn: np.ndarray, start: int) -> int:
    """Column with the largest norm among start.. ; near-ties go to the lowest index."""
    seg = vn[start:]
    mx = seg.max()
    cand = np.nonzero(seg >= mx * (1.0 - TIE_RTOL))[0]
    return start + int(cand[0])


def cpqr(Y: np.ndarray, eps: float):
    """Householder QR with column pivoting of Y (m x e), stopped at the first step i whose
    diagonal satisfies |R_ii| <= eps |R_00| (relative truncation; eps=0 never truncates
    except on an exactly zero column).

    Returns (perm, k, R) where perm lists the column order (first k = skeleton) and R holds
    the k x e upper trapezoid [R_1 R_2] in the permuted order.
    """
    Y = np.array(Y, dtype=np.float64, copy=True)
    m, e = Y.shape
    perm = np.arange(e)
    if m == 0 or e == 0:
        return perm, 0, np.zeros((0, e))
    vn1 = np.sqrt(np.sum(Y * Y, axis=0))
    vn2 = vn1.copy()
    ref = 0.0
    k = min(m, e)
    for i in range(min(m, e)):
        p = _pivot(vn1, i)
        if p != i:
            Y[:, [i, p]] = Y[:, [p, i]]
            perm[[i, p]] = perm[[p, i]]
            vn1[[i, p]] = vn1[[p, i]]
            vn2[[i, p]] = vn2[[p, i]]
        x = Y[i:, i]
        normx = float(np.sqrt(x @ x))
        if i == 0:
            ref = normx
            if ref == 0.0:
                k = 0
                break
        if normx <= eps * ref or normx == 0.0:
            k = i
            break
        alpha = -normx if x[0] >= 0 else normx
        v = x.copy()
        v[0] -= alpha
        vv = float(v @ v)
        if i + 1 < e and vv > 0.0:
            Y[i:, i + 1:] -= np.outer(v, (2.0 / vv) * (v @ Y[i:, i + 1:]))
        Y[i, i] = alpha
        Y[i + 1:, i] = 0.0
        for j in range(i + 1, e):           # norm downdate with recomputation guard
            if vn1[j] == 0.0:
                continue
            temp = 1.0 - (abs(Y[i, j]) / vn1[j]) ** 2
            temp = max(temp, 0.0)
            temp2 = temp * (vn1[j] / vn2[j]) ** 2
            if temp2 <= TOL3Z:
                vn1[j] = float(np.sqrt(Y[i + 1:, j] @ Y[i + 1:, j]))
                vn2[j] = vn1[j]
            else:
                vn1[j] *= np.sqrt(temp)
    R = np.triu(Y[:k, :])
    return perm, k, R


def interp_decomp(Y: np.ndarray, eps: float):
    """ID of Eq. (RRQR 2): returns (perm, k, T) with Y[:, perm[k:]] ~= Y[:, perm[:k]] T."""
    perm, k, R = cpqr(Y, eps)
    e = Y.shape[1]
    if k == 0:
        return perm, 0, np.zeros((0, e))
    T = solve_upper(R[:k, :k], R[:k, k:])
    return perm, k, T
