"""Philox4x32-10 and the Gaussian sampling matrix G of the hybrid sketch (Sec. 4.2.3, Eq. (Phi)).

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): a 4x32-bit counter is mixed with a
2x32-bit key by ten rounds of two 32x32->64 multiplications; the key is advanced by the
Weyl constants between rounds.  Written here from that published definition.

Entry of G (the reading of the paper used by this project; the paper only says "a Gaussian
random matrix"): for level ``l``, segment id ``sid``, sketch row ``r`` and far row labelled by
its grid node ``v`` and half ``t`` (t=0 for a row of A_{n,i}, t=1 for a row of A_{i,n}^T),
    counter = (r div 4, v, 2*l + t, sid),   key = (seed mod 2^32, seed div 2^32 mod 2^32);
the four output words give u1..u4 in (0,1) as odd multiples of 2^-24, and Box-Muller turns
each pair into two independent standard normals:
    z0 = R1 cos(2 pi u2), z1 = R1 sin(2 pi u2), z2 = R2 cos(2 pi u4), z3 = R2 sin(2 pi u4),
    R1 = sqrt(-2 log u1), R2 = sqrt(-2 log u3)
(float32, the platform's own log/sqrt/cos/sin); row r takes z_(r mod 4).  One counter thus
serves four consecutive rows.  Because each entry is addressed by (r, v, t), the sketch does
not depend on the order in which far rows are enumerated.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_SH = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Inputs are integer arrays/scalars (< 2^32); returns four
    uint64 arrays holding the 32-bit output words."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0          # exact: both factors < 2^32, product < 2^64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _SH, p0 & _MASK
        hi1, lo1 = p1 >> _SH, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
    return c0, c1, c2, c3


def _unit_f32(x):
    """(0,1) float32 from a 32-bit word: ((x >> 9) * 2 + 1) * 2^-24, exact in float32."""
    return (((np.asarray(x, dtype=np.uint64) >> np.uint64(9)) * np.uint64(2) + np.uint64(1))
            .astype(np.float32) * np.float32(2.0 ** -24))


def gaussian4_f32(c0, c1, c2, c3, seed: int):
    """Four Box-Muller normals in float32 per counter (last axis: z0..z3), two from each pair
    of Philox output words."""
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    x = philox4x32_10(c0, c1, c2, c3, k0, k1)
    u = [_unit_f32(w) for w in x]
    two_pi = np.float32(6.283185307179586)
    r1 = np.sqrt(np.float32(-2.0) * np.log(u[0]))
    r2 = np.sqrt(np.float32(-2.0) * np.log(u[2]))
    a1 = two_pi * u[1]
    a2 = two_pi * u[3]
    return np.stack([r1 * np.cos(a1), r1 * np.sin(a1), r2 * np.cos(a2), r2 * np.sin(a2)], axis=-1).astype(np.float32)


def sketch_matrix(seed: int, level: int, sid: int, h: int, far_nodes, far_half) -> np.ndarray:
    """G (h x |F|, float64 holding float32 values) for one segment: column f belongs to the
    far row with grid node far_nodes[f] and half far_half[f]."""
    far_nodes = np.asarray(far_nodes, dtype=np.int64)
    far_half = np.asarray(far_half, dtype=np.int64)
    r = np.arange(h, dtype=np.int64)[:, None]
    v = far_nodes[None, :]
    t = far_half[None, :]
    c0 = np.broadcast_to(r // 4, (h, far_nodes.size))
    c1 = np.broadcast_to(v, (h, far_nodes.size))
    c2 = np.broadcast_to(2 * level + t, (h, far_nodes.size))
    c3 = np.full((h, far_nodes.size), sid, dtype=np.int64)
    z = gaussian4_f32(c0, c1, c2, c3, seed)
    comp = np.broadcast_to(r % 4, (h, far_nodes.size))
    return np.take_along_axis(z, comp[..., None], axis=-1)[..., 0].astype(np.float64)
