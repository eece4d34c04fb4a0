"""Learned rank predictor, oracle side (test infrastructure, like the rest of ``oracle/``).

The paper finds each segment's rank with the adaptive randomized ID (Sec. 4.2.3: the sketch
has h = k + p rows, p = 5, but k is only known after the ID).  This project adds a small
network that predicts k and the one-pass sketch size from cheap features of the segment, so
that the randomized range finder can run once; the adaptive ID stays as the fallback and
judges every prediction by the measured ID error.  None of this is in the paper: every
definition below is this project's, and the CUDA path implements the same definitions.

Features of a segment (16 values, FP64), where n are its neighbour unknowns, N / F the near /
far ones (Sec. 4.2.3, hybrid sampling), u runs over the segment's grid nodes and
d_u = |A_uu|, s_u = sum_{j != u} |A_uj| are taken from the original matrix:
   0  depth below the finest level, L - l
   1  log2 e (unknowns of the segment)
   2  log2(1 + |n|)
   3  |N| (near neighbour nodes)
   4  log2(1 + |F|) (far neighbour nodes)
   5  min_u log d_u - mean_u log d_u
   6  max_u log d_u - mean_u log d_u
   7  std_u log d_u (population)
   8  mean_u log(d_u / s_u)                       (0 for a node with s_u = 0)
   9  mean_u |sum_j A_uj| / d_u                   (shift, e.g. the k^2 term of Helmholtz)
  10  mean_u sum_{j!=u}|A_uj - A_ju| / sum_{j!=u}(|A_uj| + |A_ju|)   (convection)
  11-15  probe decay above the tolerance: log10 max(|R_jj| / |R_00|, 1e-16) - log10 eps for
         j = 1, 2, 3, 5, 7, where R is the column-pivoted QR (no truncation) of the PROBE x e
         probe G_8 B_F and G_8 holds the first PROBE rows of the sketch matrix
         (``philox.sketch_matrix``); j >= min(PROBE, e), or R_00 = 0, takes the ratio 1e-16.
         Measuring the decay from the truncation level lets one network serve several eps.
Natural logarithms except where log2 / log10 is written.

Network: x -> z = (x - mu) * isd -> a = W1 z + b1 (64) -> h = max(a, 0) -> o = W2 h + b2 (2).
Parameters are one float32 vector: W1 (64 x 16, row-major) | b1 | W2 (2 x 64) | b2.
 * Training (FP32 on the GPU, FP64 here): loss = sum_{s,k} (o_sk - y_sk)^2 / (2 n) over a
   batch of n rows; Adam (beta1 0.9, beta2 0.999, eps 1e-8) over consecutive batches.
 * Inference in BF16: the parameters and z are rounded to bfloat16 (round to nearest even),
   the hidden units accumulate in float32 over i = 0..15 in order, h is rounded to bfloat16,
   the outputs accumulate over j = 0..63 in order.  A product of two bfloat16 values is
   exact in float32, so a fused multiply-add gives the same sums as a multiply then an add.
 * Targets: y0 = log2(1 + k), y1 = log2(min(|F_rows|, k + p)) with |F_rows| the far rows of
   B (far nodes times the number of halves of B) and k the rank the adaptive ID found.
 * Sketch size: h = max(ceil(2^o1 (1 + m)), ceil((2^o0 - 1)(1 + m)) + p), clamped to
   [1, min(|F_rows|, max(h0, 2 (e + p)))]; m is a safety margin (default 0.35); the outputs
   are clamped to [-30, 30] first.
 * Acceptance of the one-pass ID: k <= h - p and ||B_r - B_s T||_F <= 10 eps ||B||_F on the
   exact B; otherwise the adaptive schedule continues from h <- min(2h, |F_rows|,
   max(h0, 2 (e + p))) (at that bound k <= e < h - p, so the schedule ends).
The predictor is used for a segment only when the adaptive method would sketch it more than
once, the probe fits and the segment is not too large: |F_rows| > max(h0, PROBE),
e + p > 2 h0 (smaller segments are sketched once with h = 2 h0 >= e + p, the rank bound) and
e <= EMAX.
"""
from __future__ import annotations

import math

import numpy as np

from .dense import cpqr

NFEAT = 16
NHID = 64
NOUT = 2
NPARAM = NHID * NFEAT + NHID + NOUT * NHID + NOUT   # 1218
PROBE = 8
EMAX = 128
DECAY_J = (1, 2, 3, 5, 7)
DECAY_FLOOR = -16.0
MARGIN = 0.35
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


# ------------------------------------------------------------------ parameters
def unpack(params):
    """Views (W1, b1, W2, b2) of a parameter vector."""
    p = np.asarray(params)
    o = 0
    W1 = p[o:o + NHID * NFEAT].reshape(NHID, NFEAT); o += NHID * NFEAT
    b1 = p[o:o + NHID]; o += NHID
    W2 = p[o:o + NOUT * NHID].reshape(NOUT, NHID); o += NOUT * NHID
    b2 = p[o:o + NOUT]
    return W1, b1, W2, b2


def pack(W1, b1, W2, b2, dtype=np.float64):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2)]).astype(dtype)


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases (float32): the seeded draw of ``workloads``, an input
    to both sides."""
    from workloads import predictor_init_params
    return predictor_init_params(seed, NFEAT, NHID, NOUT)


def fit_norm(X):
    """Feature standardisation: mean and 1/std per column (1 where std < 1e-6), float32."""
    X = np.asarray(X, dtype=np.float64)
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    isd = np.where(sd < 1e-6, 1.0, 1.0 / np.where(sd < 1e-6, 1.0, sd))
    return mu.astype(np.float32), isd.astype(np.float32)


# ------------------------------------------------------------------ bfloat16
def bf16(x):
    """Round float32 values to the nearest bfloat16 (ties to even); returned as float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)) << np.uint64(16)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).reshape(a.shape)


def infer_bf16(params, mu, isd, X):
    """BF16 inference of the rows of X (n x 16); returns float32 outputs (n x 2)."""
    W1, b1, W2, b2 = (bf16(np.asarray(t, dtype=np.float32)) for t in unpack(np.asarray(params, np.float32)))
    X32 = np.asarray(X, dtype=np.float64).astype(np.float32)
    n = X32.shape[0]
    z = bf16((X32 - np.asarray(mu, np.float32)[None, :]) * np.asarray(isd, np.float32)[None, :])
    acc = np.broadcast_to(b1[None, :], (n, NHID)).astype(np.float32)
    for i in range(NFEAT):                       # float32 sums in the order i = 0..15
        acc = (acc + W1[None, :, i] * z[:, i:i + 1]).astype(np.float32)
    h = bf16(np.maximum(acc, np.float32(0.0)))
    out = np.broadcast_to(b2[None, :], (n, NOUT)).astype(np.float32)
    for j in range(NHID):
        out = (out + W2[None, :, j] * h[:, j:j + 1]).astype(np.float32)
    return out


def sketch_size(o, nF_rows: int, e: int, p: int, h0: int, margin: float) -> int:
    """One-pass sketch size from the network outputs (float32 arithmetic, as on the GPU)."""
    o0 = np.float32(min(max(float(o[0]), -30.0), 30.0)) if math.isfinite(float(o[0])) else np.float32(-30.0)
    o1 = np.float32(min(max(float(o[1]), -30.0), 30.0)) if math.isfinite(float(o[1])) else np.float32(-30.0)
    m1 = np.float32(1.0) + np.float32(margin)
    hh = math.ceil(float(np.float32(np.exp2(o1)) * m1))
    kh = math.ceil(float((np.float32(np.exp2(o0)) - np.float32(1.0)) * m1)) + p
    h = max(hh, kh, 1)
    return int(min(h, nF_rows, max(h0, 2 * (e + p))))


# ------------------------------------------------------------------ training (FP64)
def forward(params, mu, isd, X):
    W1, b1, W2, b2 = (np.asarray(t, np.float64) for t in unpack(np.asarray(params, np.float64)))
    z = (np.asarray(X, np.float64) - np.asarray(mu, np.float64)) * np.asarray(isd, np.float64)
    a = z @ W1.T + b1
    h = np.maximum(a, 0.0)
    o = h @ W2.T + b2
    return z, a, h, o


def loss_grad(params, mu, isd, X, Y):
    """Loss sum (o - y)^2 / (2n) and its gradient with respect to the parameters (FP64)."""
    W1, b1, W2, b2 = (np.asarray(t, np.float64) for t in unpack(np.asarray(params, np.float64)))
    z, a, h, o = forward(params, mu, isd, X)
    n = z.shape[0]
    r = o - np.asarray(Y, np.float64)
    loss = float(np.sum(r * r) / (2.0 * n))
    dO = r / n
    gW2 = dO.T @ h
    gb2 = dO.sum(axis=0)
    da = (dO @ W2) * (a > 0.0)
    gW1 = da.T @ z
    gb1 = da.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2)


def adam_step(params, m, v, g, t: int, lr: float):
    """One Adam update (t counts from 1); returns new (params, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * g
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * g * g
    mh = m / (1.0 - ADAM_B1 ** t)
    vh = v / (1.0 - ADAM_B2 ** t)
    return params - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def train(params, mu, isd, X, Y, epochs: int, batch: int, lr: float):
    """Adam over consecutive batches of the rows, ``epochs`` times; returns (params, losses)."""
    p = np.asarray(params, np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    t = 0
    losses = []
    n = len(X)
    for _ in range(epochs):
        tot = 0.0
        for b0 in range(0, n, batch):
            xb, yb = X[b0:b0 + batch], Y[b0:b0 + batch]
            loss, g = loss_grad(p, mu, isd, xb, yb)
            tot += loss * len(xb)
            t += 1
            p, m, v = adam_step(p, m, v, g, t, lr)
        losses.append(tot / n)
    return p, losses


def targets(k: int, nF_rows: int, p: int):
    return np.array([math.log2(1 + k), math.log2(max(1, min(nF_rows, k + p)))])


# ------------------------------------------------------------------ features
def coefficient_stats(A, seg_nodes):
    """Features 5-10 from the original CSR matrix at the segment's grid nodes."""
    logd, dom, shift, asym = [], [], [], []
    for u in np.asarray(seg_nodes, dtype=np.int64):
        s, e = A.indptr[u], A.indptr[u + 1]
        d = 0.0
        off = 0.0
        rs = 0.0
        num = den = 0.0
        for j, a in zip(A.indices[s:e], A.data[s:e]):
            rs += a
            if j == u:
                d += a
                continue
            off += abs(a)
            # A_ju from row j
            aj = 0.0
            for jj, b in zip(A.indices[A.indptr[j]:A.indptr[j + 1]], A.data[A.indptr[j]:A.indptr[j + 1]]):
                if jj == u:
                    aj += b
            num += abs(a - aj)
            den += abs(a) + abs(aj)
        d = abs(d)
        ld = math.log(d) if d > 0.0 else math.log(1e-300)
        logd.append(ld)
        dom.append(math.log(d / off) if off > 0.0 and d > 0.0 else 0.0)
        shift.append(abs(rs) / d if d > 0.0 else 0.0)
        asym.append(num / den if den > 0.0 else 0.0)
    logd = np.array(logd)
    mean = logd.mean()
    return [logd.min() - mean, logd.max() - mean, float(np.sqrt(np.mean((logd - mean) ** 2))),
            float(np.mean(dom)), float(np.mean(shift)), float(np.mean(asym))]


def probe_decay(P, eps: float):
    """Features 11-15 from the probe matrix P (PROBE x e) and the ID tolerance."""
    e = P.shape[1]
    _, k, R = cpqr(P, 0.0)
    diag = np.zeros(min(P.shape[0], e))
    for i in range(k):
        diag[i] = abs(R[i, i])
    le = math.log10(eps)
    out = []
    for j in DECAY_J:
        if j >= diag.size or diag[0] == 0.0:
            out.append(DECAY_FLOOR - le)
        else:
            out.append(math.log10(max(diag[j] / diag[0], 1e-16)) - le)
    return out


def features(A, L: int, l: int, seg_nodes, n_nbr: int, n_near: int, n_far: int, probe, eps: float):
    x = [float(L - l), math.log2(len(seg_nodes)), math.log2(1 + n_nbr), float(n_near),
         math.log2(1 + n_far)]
    x += coefficient_stats(A, seg_nodes)
    x += probe_decay(probe, eps)
    return np.array(x, dtype=np.float64)


def id_error_ok(B, perm, k: int, T, eps: float) -> bool:
    """Measured ID error test: ||B_r - B_s T||_F <= 10 eps ||B||_F."""
    Bs = B[:, perm[:k]]
    Br = B[:, perm[k:]]
    res = Br - Bs @ T if k > 0 else Br
    return float(np.linalg.norm(res)) <= 10.0 * eps * float(np.linalg.norm(B))
