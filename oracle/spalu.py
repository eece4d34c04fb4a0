"""Oracle of the spaLU factorization (Sec. 4.3, Alg. 2) and of its solve (Eq. (WV)).

The Schur complement A^(l) is held as a dictionary of dense blocks between *groups* of
unknowns (segments, their skeleton / remainder parts, and junctions); every step below
reads and writes that global Schur complement directly.

Readings of the paper used here (the paper is silent or loose on these points):
  * Neighbours of a segment (Sec. 2.3.2): every current unknown on the boundary of the two
    depth-l boxes adjacent to it (other sides and corners), coupled or not.
  * Stacking (Sec. 4.5, Eq. (ID [A_ni; A_in])): B = [A_{n,i}; A_{i,n}^T] unless the caller
    declares A symmetric, in which case B = A_{n,i}; one ID gives L_t = U_t^T.
  * Hybrid sampling (Sec. 4.2.3, Eq. (Phi)): near rows are the neighbours within Chebyshev
    distance ``near_radius`` (2) of the segment (this includes both end junctions); the
    far rows are replaced by G B_F / sqrt(h) with G from ``philox.sketch_matrix``; when the
    far block has no more than h rows it is taken whole (Phi = I).
  * Sketch size (h = k + p, p = 5 in Sec. 4.2.3; k unknown in advance): the rank is at most
    the segment's size e, so a segment with e + p <= 2 h0 is sketched once with
    h = min(|F|, 2 h0, max(h0, 2 (e + p))) (the size the adaptive schedule below reaches at its
    second pass, within the schedule's own cap), and k <= e <= h - p holds at once (or h = |F|
    and the far block is taken whole); a larger one starts with h = min(|F|, h0 = 16), and after
    the ID, while k > h - p and h < |F|, h doubles (capped at |F|) and the sketch and the ID
    are redone.
  * Truncation (Sec. 4.1): relative, the first k with |R_{k+1,k+1}| <= eps |R_{11}|.
    eps = 0 skips sparsification altogether (k = e), which makes the method exact block LU.
  * Order inside a level (Alg. 2 loops "for each segment"): every ID of level l is taken
    from A^(l) as it stands at the start of the level; then all transforms are applied,
    blocks coupling a remainder to its neighbours are dropped (they are O(eps)), then all
    remainders are eliminated, then the level-l separators (their skeletons).
  * Merge (Sec. 4.3, E_(l)): the unknowns of a side of a depth-(l-1) box are, in order of
    increasing coordinate of the pieces, [skeleton of child side 1, junction, skeleton of
    child side 2], each skeleton in the order chosen by the column pivoting.
"""
from __future__ import annotations

import math
from collections import defaultdict
from dataclasses import dataclass, field

import numpy as np

from .dense import gepp, interp_decomp, lu_solve
from . import flops as fl
from .nd import NestedDissection, box_corners, chebyshev_to_segment, _sides
from .philox import sketch_matrix
from . import predictor as pred


@dataclass
class Options:
    eps: float = 1e-8
    symmetric: bool = False
    p_oversample: int = 5
    near_radius: int = 2          # -1: no near rows (pure randomized sampling, Sec. 4.2.1)
    h0: int = 16
    seed: int = 0
    # learned rank predictor (not in the paper; see oracle/predictor.py): a dict with
    # "params", "mu", "isd" and optionally "margin"; and a list that receives one
    # (features, k, far rows, e, l) tuple per segment the predictor applies to
    predictor: dict | None = None
    record: list | None = None


@dataclass
class Elim:
    """Block elimination of unknowns p against their neighbours q (one factor of
    L_(l) / U_(l)): forward b_q -= A_qp A_pp^{-1} b_p; backward
    x_p = A_pp^{-1} (b_p - A_pq x_q)."""
    p: np.ndarray
    q: np.ndarray
    lu: np.ndarray
    piv: np.ndarray
    Aqp: np.ndarray
    Apq: np.ndarray


@dataclass
class Sparsify:
    """Sparsification of one segment, U_t and L_t = U_t^T of Eq. (B): forward
    b_r -= T^T b_s; backward x_s -= T x_r."""
    sk: np.ndarray
    r: np.ndarray
    T: np.ndarray


@dataclass
class Factor:
    N: int
    tape: list
    stats: dict = field(default_factory=dict)


class _Blocks:
    """Dense blocks of the current Schur complement, keyed by (row group, column group)."""

    def __init__(self):
        self.d: dict = {}
        self.adj: dict = defaultdict(set)

    def get(self, a, b):
        return self.d.get((a, b))

    def add(self, a, b, M):
        if M.size == 0:
            return
        if (a, b) in self.d:
            self.d[(a, b)] += M
        else:
            self.d[(a, b)] = np.array(M, dtype=np.float64, copy=True)
            self.adj[a].add(b)
            self.adj[b].add(a)

    def drop_group(self, g):
        for o in list(self.adj.get(g, ())):
            self.d.pop((g, o), None)
            self.d.pop((o, g), None)
            if o != g:
                self.adj[o].discard(g)
        self.adj.pop(g, None)


def _csr_block(A, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Dense A[rows, cols] gathered from CSR."""
    col_pos = {int(c): i for i, c in enumerate(cols)}
    out = np.zeros((rows.size, cols.size))
    for i, r in enumerate(rows):
        s, e = A.indptr[r], A.indptr[r + 1]
        for c, v in zip(A.indices[s:e], A.data[s:e]):
            j = col_pos.get(int(c))
            if j is not None:
                out[i, j] += v
    return out


def factor(A, nd: NestedDissection, opts: Options = Options()) -> Factor:
    """Alg. 2: leaf-interior elimination, then for l = L..1 sparsify, eliminate, merge."""
    nx = nd.nx
    tape: list = []
    blk = _Blocks()
    nodes: dict = {}
    stats = {"levels": {}}
    L = nd.L

    # ---- groups of level L and the original couplings between separator unknowns
    if L >= 1:
        lev = nd.levels[L]
        where = {}
        for key, seg in lev.segments.items():
            g = ("S", L, key)
            nodes[g] = seg.nodes.copy()
            for pos, v in enumerate(seg.nodes):
                where[int(v)] = (g, pos)
        for c in lev.corners:
            g = ("J", c)
            nodes[g] = np.array([c], dtype=np.int64)
            where[int(c)] = (g, 0)
        acc = defaultdict(list)
        for u, (gu, pu) in where.items():
            s, e = A.indptr[u], A.indptr[u + 1]
            for v, a in zip(A.indices[s:e], A.data[s:e]):
                hit = where.get(int(v))
                if hit is not None:
                    acc[(gu, hit[0])].append((pu, hit[1], a))
        for (ga, gb), ents in acc.items():
            M = np.zeros((nodes[ga].size, nodes[gb].size))
            for i, j, a in ents:
                M[i, j] += a
            blk.add(ga, gb, M)

    # ---- leaf-interior elimination (Sec. 4.3, first step: L_(L+1), U_(L+1))
    for b in nd.leaves:
        I = np.array([x + nx * y for y in range(b.y0, b.y1 + 1) for x in range(b.x0, b.x1 + 1)],
                     dtype=np.int64)
        sides = [(("S", L, key), np.array(nl, dtype=np.int64)) for key, nl in _sides(b, nx, nd.ny)]
        D = np.concatenate([nl for _, nl in sides]) if sides else np.zeros(0, dtype=np.int64)
        A_II = _csr_block(A, I, I)
        A_ID = _csr_block(A, I, D)
        A_DI = _csr_block(A, D, I)
        lu, piv = gepp(A_II)
        if D.size:
            S = A_DI @ lu_solve(lu, piv, A_ID)
            off = np.cumsum([0] + [nl.size for _, nl in sides])
            for a, (ga, _) in enumerate(sides):
                for c, (gb, _) in enumerate(sides):
                    blk.add(ga, gb, -S[off[a]:off[a + 1], off[c]:off[c + 1]])
        tape.append(Elim(I, D, lu, piv, A_DI, A_ID))

    # ---- level loop (Alg. 2, l = L..1)
    for l in range(L, 0, -1):
        lev = nd.levels[l]
        keys = sorted(lev.segments, key=lambda k: lev.segments[k].sid)
        seg_g = {k: ("S", l, k) for k in keys}
        ids = {}
        e_max, k_max = 0, 0
        cnt = {"passes": 0, "fallbacks": 0, "predicted": 0, "flops_sparsify": 0}
        # 1. one ID per segment, all from A^(l) as it stands (Eqs. (RRQR sample), (ID [A_ni; A_in]))
        for key in keys:
            g = seg_g[key]
            e = nodes[g].size
            e_max = max(e_max, e)
            if opts.eps == 0.0:
                ids[key] = (np.arange(e), e, np.zeros((e, 0)))
                k_max = max(k_max, e)
                continue
            nbr = _neighbour_groups(lev.segments[key], l, nx, nd.ny, nodes)
            ids[key] = _segment_id(blk, g, key, nbr, nodes, l, lev.segments[key].sid, nx, opts,
                                   A, L, cnt)
            k_max = max(k_max, ids[key][1])
        for key in keys:             # transforms and remainder eliminations of this level
            e = nodes[seg_g[key]].size
            k = int(ids[key][1])
            cnt["flops_sparsify"] += fl.apply(e, k) + (fl.elim(e - k, k) if e > k else 0)
        stats["levels"][l] = {"e_max": e_max, "k_max": k_max, **cnt,
                              "ranks": [int(ids[k][1]) for k in keys],
                              "sizes": [int(nodes[seg_g[k]].size) for k in keys],
                              # index tables: segment nodes entering the level and in ID order
                              # (skeleton first, in pivot order), keyed by segment id
                              "nodes": {lev.segments[k].sid: nodes[seg_g[k]].copy() for k in keys},
                              "skel": {lev.segments[k].sid: nodes[seg_g[k]][ids[k][0]] for k in keys}}

        # 2. apply U_T^(l) A^(l) L_T^(l) (Eq. (U_T * A * LT)): transformed diagonal blocks,
        #    neighbour couplings restricted to skeletons, remainder couplings dropped.
        split = {}
        for key in keys:
            perm, k, _ = ids[key]
            split[seg_g[key]] = (("K", l, key), perm[:k], ("R", l, key), perm[k:])
        new = _Blocks()
        new_nodes = {}
        for g, nl in nodes.items():
            if g in split:
                kg, ki, rg, ri = split[g]
                if ki.size:
                    new_nodes[kg] = nl[ki]
                if ri.size:
                    new_nodes[rg] = nl[ri]
            else:
                new_nodes[g] = nl
        for (ga, gb), M in blk.d.items():
            if ga == gb and ga in split:
                continue
            ka, ia = (split[ga][0], split[ga][1]) if ga in split else (ga, np.arange(M.shape[0]))
            kb, ib = (split[gb][0], split[gb][1]) if gb in split else (gb, np.arange(M.shape[1]))
            if ia.size and ib.size:
                new.add(ka, kb, M[np.ix_(ia, ib)])
        rem = []
        for key in keys:
            g = seg_g[key]
            perm, k, T = ids[key]
            kg, _, rg, _ = split[g]
            Ass = blk.get(g, g)
            Ap = Ass[np.ix_(perm, perm)]
            A_kk, A_kr, A_rk, A_rr = Ap[:k, :k], Ap[:k, k:], Ap[k:, :k], Ap[k:, k:]
            A_kr1 = A_kr - A_kk @ T          # column operation  A_{:,r} -= A_{:,s} T
            A_rr1 = A_rr - A_rk @ T
            A_rk2 = A_rk - T.T @ A_kk        # row operation     A_{r,:} -= T^T A_{s,:}
            A_rr2 = A_rr1 - T.T @ A_kr1
            new.add(kg, kg, A_kk)
            new.add(kg, rg, A_kr1)
            new.add(rg, kg, A_rk2)
            new.add(rg, rg, A_rr2)
            r_nodes = nodes[g][perm[k:]]
            sk_nodes = nodes[g][perm[:k]]
            if r_nodes.size and sk_nodes.size:
                tape.append(Sparsify(sk_nodes, r_nodes, T.copy()))
            if r_nodes.size:
                rem.append((kg, rg, sk_nodes, r_nodes))
        blk, nodes = new, new_nodes

        # 3. eliminate remainders (Eq. (L^-1 * A * U^-1), segments of level l)
        for kg, rg, sk_nodes, r_nodes in rem:
            _eliminate(blk, rg, nodes, tape)

        # 4. eliminate the level-l separators (their skeletons)
        kps = []
        for key in lev.separators:
            kg = ("K", l, key)
            kps.append(nodes[kg].size if kg in nodes else 0)
            if kg in nodes:
                _eliminate(blk, kg, nodes, tape)

        # 5. merge skeletons into the segments of level l-1 (E_(l))
        if l > 1:
            nodes, blk = _merge(nd, l, nodes, blk)
        # work of the separator eliminations, counted against every unknown on the boundary of
        # the parent box after the merge (its sides and its existing corners)
        fm = 0
        for parent, kp in zip(lev.parents, kps):
            dP = sum(nodes[("S", l - 1, key)].size for key, _ in _sides(parent, nx, nd.ny)) if l > 1 else 0
            dP += len(box_corners(parent, nx, nd.ny)) if l > 1 else 0
            fm += fl.elim(kp, dP) if kp else 0
        stats["levels"][l]["flops_merge"] = fm

    assert not blk.d, "unknowns left after level 1"
    ks = [v["k_max"] / v["e_max"] for v in stats["levels"].values() if v["e_max"] > 0]
    stats["q_tilde"] = max(ks) if ks else 0.0
    return Factor(nd.N, tape, stats)


def _neighbour_groups(seg, l, nx, ny, nodes):
    """Groups on the boundary of the depth-l boxes adjacent to a segment, excluding it."""
    out = []
    seen = set()
    for b in seg.boxes:
        for key, _ in _sides(b, nx, ny):
            g = ("S", l, key)
            if key != seg.key and g not in seen:
                seen.add(g)
                out.append(g)
        for c in box_corners(b, nx, ny):
            g = ("J", c)
            if g not in seen:
                seen.add(g)
                out.append(g)
    return out


def _segment_id(blk, g, key, nbr, nodes, l, sid, nx, opts: Options, A=None, L=0, cnt=None):
    """Sampled ID of one segment (Secs. 4.1-4.2, 4.5): returns (perm, k, T).  With a
    predictor, the first sketch has the predicted size and is kept only if it passes the
    measured-error test; otherwise the adaptive schedule continues."""
    cnt = cnt if cnt is not None else {"passes": 0, "fallbacks": 0, "predicted": 0, "flops_sparsify": 0}
    e = nodes[g].size
    rows_n, rows_t, labels = [], [], []
    for gn in nbr:
        m = nodes[gn].size
        if m == 0:
            continue
        M1 = blk.get(gn, g)
        M2 = blk.get(g, gn)
        rows_n.append(M1 if M1 is not None else np.zeros((m, e)))
        rows_t.append(M2.T if M2 is not None else np.zeros((m, e)))
        labels.append(nodes[gn])
    if labels:
        Bn = np.vstack(rows_n)
        Bt = np.vstack(rows_t)
        vlab = np.concatenate(labels)
    else:
        Bn = Bt = np.zeros((0, e))
        vlab = np.zeros(0, dtype=np.int64)
    near = np.array([chebyshev_to_segment(key, int(v), nx) <= opts.near_radius for v in vlab],
                    dtype=bool)
    halves = [(Bn, 0)] if opts.symmetric else [(Bn, 0), (Bt, 1)]
    BN = np.vstack([Bh[near] for Bh, _ in halves]) if vlab.size else np.zeros((0, e))
    BF = np.vstack([Bh[~near] for Bh, _ in halves]) if vlab.size else np.zeros((0, e))
    f_nodes = np.concatenate([vlab[~near] for _ in halves]) if vlab.size else np.zeros(0, np.int64)
    f_half = np.concatenate([np.full(int((~near).sum()), t) for _, t in halves]) if vlab.size \
        else np.zeros(0, np.int64)
    nF = BF.shape[0]

    def ident():
        r = interp_decomp(np.vstack([BN, BF]), opts.eps)
        cnt["flops_sparsify"] += fl.qr(BN.shape[0] + nF, e, r[1])
        return r

    def done(r):
        cnt["flops_sparsify"] += fl.interp(r[1], e)
        return r

    cnt["passes"] += 1
    if nF <= opts.h0:
        return done(ident())
    p = opts.p_oversample
    h = min(nF, opts.h0)
    # rank bound: k <= e, so a segment with e + p <= 2 h0 is sketched once with h = 2 h0 (the
    # size the adaptive schedule reaches at its second pass), and that pass always stands
    small = e + p <= 2 * opts.h0
    if small:
        h = min(nF, 2 * opts.h0, max(opts.h0, 2 * (e + p)))
    use_pred = (opts.predictor is not None or opts.record is not None) and A is not None \
        and nF > max(opts.h0, pred.PROBE) and e <= pred.EMAX and not small
    predicted = False
    if use_pred:
        probe = sketch_matrix(opts.seed, l, sid, pred.PROBE, f_nodes, f_half) @ BF
        x = pred.features(A, L, l, nodes[g], int(vlab.size), int(near.sum()), int((~near).sum()), probe,
                          opts.eps)
        if opts.predictor is not None:
            pr = opts.predictor
            o = pred.infer_bf16(pr["params"], pr["mu"], pr["isd"], x[None, :])[0]
            h = pred.sketch_size(o, nF, e, p, opts.h0, pr.get("margin", pred.MARGIN))
            predicted = True
            cnt["predicted"] += 1
    Bx = Bn if opts.symmetric else np.vstack([Bn, Bt])      # the exact B of Eq. (ID [A_ni; A_in])
    while True:
        if h >= nF:
            res = ident()
            break
        G = sketch_matrix(opts.seed, l, sid, h, f_nodes, f_half)
        Y = np.vstack([BN, (G @ BF) / math.sqrt(h)])
        perm, k, T = interp_decomp(Y, opts.eps)
        # work count: a pass that may still double h only has to establish k > h - p, so its
        # QR counts min(k, h - p + 1) steps (the library stops there; the results are the same)
        cnt["flops_sparsify"] += fl.sketch(h, nF, e) + fl.qr(Y.shape[0], e, min(k, max(1, h - p + 1)))
        if predicted:
            predicted = False
            if k <= h - p and pred.id_error_ok(Bx, perm, k, T, opts.eps):
                res = (perm, k, T)
                break
            cnt["fallbacks"] += 1
            cnt["passes"] += 1
            h = min(2 * h, nF, max(opts.h0, 2 * (e + p)))
            continue
        if k > h - p and h < nF:
            cnt["passes"] += 1
            h = min(2 * h, nF, max(opts.h0, 2 * (e + p)))   # binds only after a prediction
            continue
        res = (perm, k, T)
        break
    if use_pred and opts.record is not None:
        opts.record.append((x, int(res[1]), int(nF), int(e), int(l)))
    return done(res)


def _eliminate(blk: _Blocks, p, nodes, tape):
    """Eliminate group p against every group coupled to it; record the Elim op."""
    nbrs = sorted((o for o in blk.adj.get(p, ()) if o != p), key=repr)
    App = blk.get(p, p)
    lu, piv = gepp(App)
    npv = nodes[p].size
    qs = [nodes[o] for o in nbrs]
    sizes = [q.size for q in qs]
    off = np.cumsum([0] + sizes)
    Aqp = np.zeros((off[-1], npv))
    Apq = np.zeros((npv, off[-1]))
    for i, o in enumerate(nbrs):
        M = blk.get(o, p)
        if M is not None:
            Aqp[off[i]:off[i + 1]] = M
        M = blk.get(p, o)
        if M is not None:
            Apq[:, off[i]:off[i + 1]] = M
    if nbrs:
        S = Aqp @ lu_solve(lu, piv, Apq)
        for i, a in enumerate(nbrs):
            for j, b in enumerate(nbrs):
                blk.add(a, b, -S[off[i]:off[i + 1], off[j]:off[j + 1]])
    q = np.concatenate(qs) if qs else np.zeros(0, dtype=np.int64)
    tape.append(Elim(nodes[p].copy(), q, lu, piv, Aqp, Apq))
    blk.drop_group(p)
    del nodes[p]


def _merge(nd: NestedDissection, l: int, nodes, blk: _Blocks):
    """Regroup the unknowns left after level l into the segments and junctions of level l-1."""
    nx = nd.nx
    up = nd.levels[l - 1]
    by_line = defaultdict(list)
    for key in up.segments:
        by_line[(key[0], key[1])].append(key)
    up_corners = set(up.corners)

    def host(orient, line, lo, hi):
        for k in by_line.get((orient, line), ()):
            if k[2] <= lo and hi <= k[3]:
                return k
        return None

    pieces = defaultdict(list)      # level-(l-1) key -> [(start coordinate, old group)]
    keep = {}
    for g, nl in nodes.items():
        if g[0] == "K":
            key = g[2]
            k2 = host(key[0], key[1], key[2], key[3])
            assert k2 is not None
            pieces[k2].append((key[2], g))
        elif g[0] == "J":
            c = g[1]
            if c in up_corners:
                keep[g] = g
                continue
            x, y = c % nx, c // nx
            k2 = host("H", y, x, x) or host("V", x, y, y)
            assert k2 is not None
            pieces[k2].append((x if k2[0] == "H" else y, g))
        else:
            raise AssertionError(f"unexpected group {g}")
    to_new = {}
    new_nodes = {}
    for k2, lst in pieces.items():
        lst.sort(key=lambda t: t[0])
        G = ("S", l - 1, k2)
        off = 0
        parts = []
        for _, g in lst:
            to_new[g] = (G, off)
            off += nodes[g].size
            parts.append(nodes[g])
        new_nodes[G] = np.concatenate(parts)
    for g in keep:
        to_new[g] = (g, 0)
        new_nodes[g] = nodes[g]
    sizes = {G: nl.size for G, nl in new_nodes.items()}
    acc: dict = {}
    for (ga, gb), M in blk.d.items():
        Ga, oa = to_new[ga]
        Gb, ob = to_new[gb]
        if (Ga, Gb) not in acc:
            acc[(Ga, Gb)] = np.zeros((sizes[Ga], sizes[Gb]))
        acc[(Ga, Gb)][oa:oa + M.shape[0], ob:ob + M.shape[1]] += M
    new = _Blocks()
    for (Ga, Gb), M in acc.items():
        new.add(Ga, Gb, M)
    return new_nodes, new


def solve(F: Factor, B: np.ndarray) -> np.ndarray:
    """Apply W~ (forward, in factorization order) then V~ (backward, reversed): Eq. (WV)."""
    v = np.array(B, dtype=np.float64, copy=True)
    squeeze = v.ndim == 1
    if squeeze:
        v = v[:, None]
    for op in F.tape:
        if isinstance(op, Elim):
            if op.q.size:
                t = lu_solve(op.lu, op.piv, v[op.p])
                v[op.q] -= op.Aqp @ t
        else:
            v[op.r] -= op.T.T @ v[op.sk]
    for op in reversed(F.tape):
        if isinstance(op, Elim):
            rhs = v[op.p] - (op.Apq @ v[op.q] if op.q.size else 0.0)
            v[op.p] = lu_solve(op.lu, op.piv, rhs)
        else:
            v[op.sk] -= op.T @ v[op.r]
    return v[:, 0] if squeeze else v
