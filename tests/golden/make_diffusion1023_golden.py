"""Write the 1023 x 1023 diffusion golden file from the CPU oracle (and nothing else).

The problem is the full-size variable-coefficient workload (a = exp(GRF), length 0.05,
variance 1) with seed 1 and one standard-normal right-hand side; the oracle factors it at
eps_ID = 1e-8 (FP64, adaptive ID) and solves.  Stored: the solution's 2-norm, max-norm and
sum, the input's digest (sum and 2-norm of the matrix values, norm of B), its values at a fixed sample of unknowns (one interior node of every leaf box, every
node of the level-1 separator, 1024 further separator nodes), and per level the oracle's
largest segment, largest rank and work counts.  The vector itself (8 MB) is not stored.

    python tests/golden/make_diffusion1023_golden.py     # about three minutes on one core
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle.nd import nested_dissection  # noqa: E402
from oracle.spalu import Options, factor, solve  # noqa: E402

N_SIDE, SEED, EPS = 1023, 1, 1e-8
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "diffusion1023_seed1_eps1e-8.json")


def sample_indices(nd) -> np.ndarray:
    rng = np.random.default_rng(2024)
    n = nd.nx
    idx = []
    for b in nd.leaves:                       # one interior node per leaf box
        x = int(rng.integers(b.x0, b.x1 + 1))
        y = int(rng.integers(b.y0, b.y1 + 1))
        idx.append(x + n * y)
    idx.extend(int(v) for v in nd.seps[1][0][1])           # the whole level-1 separator
    seps = np.concatenate([v for l in range(2, nd.L + 1) for _, v in nd.seps[l]])
    idx.extend(int(v) for v in rng.choice(seps, size=1024, replace=False))
    return np.array(sorted(set(idx)), dtype=np.int64)


def main():
    t0 = time.time()
    P = W.make_problem("diffusion", N_SIDE, seed=SEED, nrhs=1)
    nd = nested_dissection(N_SIDE, N_SIDE)
    F = factor(P.A, nd, Options(eps=EPS, symmetric=True))
    x = solve(F, P.B)[:, 0]
    idx = sample_indices(nd)
    out = {
        "what": "oracle solution of diffusion 1023x1023 (a=exp(GRF l=0.05 var=1), seed 1, 1 RHS), "
                "eps_ID=1e-8, FP64 adaptive ID",
        "n": N_SIDE, "seed": SEED, "eps_id": EPS, "nrhs": 1,
        "norm2": float(np.linalg.norm(x)), "norminf": float(np.max(np.abs(x))), "sum": float(x.sum()),
        "b_norm2": float(np.linalg.norm(P.B[:, 0])),
        "a_sum": float(P.A.data.sum()), "a_norm2": float(np.linalg.norm(P.A.data)),
        "index": idx.tolist(), "value": [float(v) for v in x[idx]],
        "levels": {str(l): {k: int(v[k]) for k in ("e_max", "k_max", "flops_sparsify", "flops_merge", "passes")}
                   for l, v in F.stats["levels"].items()},
        "oracle_seconds": round(time.time() - t0, 1),
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print(OUT, out["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
