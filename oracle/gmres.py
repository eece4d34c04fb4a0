"""Right-preconditioned restarted GMRES (Saad & Schultz 1986) with modified Gram-Schmidt
and Givens rotations; the preconditioner is the spaLU solve.  One independent run per
right-hand side column, each stopped when ||b - A x||_2 <= tol ||b||_2."""
from __future__ import annotations

import numpy as np


def gmres(matvec, psolve, b: np.ndarray, x0: np.ndarray, m: int = 30, tol: float = 1e-10,
          maxit: int = 200):
    """Returns (x, iterations, relative residual)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return np.zeros_like(x), 0, 0.0
    r = b - matvec(x)
    beta = float(np.linalg.norm(r))
    it = 0
    while beta > tol * bn and it < maxit:
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        j_last = -1
        for j in range(m):
            z = psolve(V[j])
            Z.append(z)
            w = matvec(z)
            for i in range(j + 1):
                H[i, j] = float(w @ V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = float(np.hypot(H[j, j], H[j + 1, j]))
            cs[j], sn[j] = (1.0, 0.0) if den == 0 else (H[j, j] / den, H[j + 1, j] / den)
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_last = j
            if abs(g[j + 1]) <= tol * bn or it >= maxit:
                break
        k = j_last + 1
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
        r = b - matvec(x)
        beta = float(np.linalg.norm(r))
    return x, it, beta / bn
