"""Comparison helpers of the parity tests: a solution against its reference, whole and entry
by entry.

Both bars must hold: the relative 2-norm difference over all columns, and for every column the
largest entry-wise difference relative to that column's largest reference entry, so that an
error confined to one leaf or one coarse segment cannot hide inside a global norm.
"""
import numpy as np


def rel_errors(X, Xo):
    """(norm-wise relative difference, largest per-column max |x - x_o| / max |x_o|)."""
    X = np.asarray(X, dtype=np.float64)
    Xo = np.asarray(Xo, dtype=np.float64)
    assert X.shape == Xo.shape, (X.shape, Xo.shape)
    if X.ndim == 1:
        X, Xo = X[:, None], Xo[:, None]
    nrm = np.linalg.norm(X - Xo) / max(np.linalg.norm(Xo), 1e-300)
    inf = np.max(np.abs(Xo), axis=0)
    ent = np.max(np.abs(X - Xo), axis=0) / np.where(inf > 0, inf, 1.0)
    return float(nrm), float(ent.max(initial=0.0))


def assert_close(X, Xo, tol, what=""):
    nrm, ent = rel_errors(X, Xo)
    assert nrm <= tol and ent <= tol, f"{what}: norm-wise {nrm:.3e}, entry-wise {ent:.3e}, bar {tol:.1e}"
    return nrm, ent
