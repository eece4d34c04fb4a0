#!/usr/bin/env python
"""Benchmark: factor + solve DOF/s of the spaLU fast direct solver on one GB300.

Step = one numeric factorization of the 1023 x 1023 variable-coefficient diffusion matrix
(a = exp(GRF), squared-exponential covariance with length 0.05, variance 1), the direct
solve of 16 standard-normal right-hand sides and GMRES refinement of every column to a
relative residual <= 1e-10.  value = N / (T_factor + T_solve+refine), summed over ranks.
The headline path is mixed precision with the learned rank predictor, trained on the GPU
before the timed region from adaptive-ID records of smaller problems (n <= 511); the plain
FP64 form (adaptive ID) is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank factors its own instance (seed + rank): the problems are
independent, so there is no data-path collective and scaling is weak.  --impl reference
times the CPU oracle (the plain FP64 restatement of the method) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# the CPU oracle leg is reported as single-threaded: keep numpy's BLAS on one thread
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

METRIC = "factor+solve DOF/s at N≈1M, mixed+learned vs plain FP64 GPU @1e-10 residual"
N_SIDE = 1023
NRHS = 16
# relative margin of the learned sketch size h = (k^ + p)(1 + margin): measured faster than the
# library default 0.35 at eps_ID 4e-7 .. 5e-7 (fewer fallbacks outweigh the larger sketches)
PRED_MARGIN = 0.7
EPS_ID = 1e-8
FP64_FLOP_PER_CLK_SM = 4          # 2 FP64 FMA per clock per SM on GB300 (measured: 1.19 TFLOP/s)
FP32_FLOP_PER_CLK_SM = 256        # 128 FP32 lanes x FMA per clock per SM
N_SM = 152
SM_MAX_MHZ = 2070.0
# training problems of the predictor (kind, n, seed): the families of the method at n <= 511
TRAIN_SET = [("diffusion", 255, 101), ("diffusion", 255, 102), ("diffusion", 511, 103),
             ("laplace", 255, 104), ("helmholtz", 255, 105), ("convdiff", 255, 106)]


def leaf_algorithmic_flops() -> float:
    """FP64 FLOPs of one leaf elimination: band LU of the 225 x 225 interior (bandwidths
    15/15, no pivot fill) and 60 band solves for the Schur complement onto the sides."""
    n, b = 225, 15
    lu = 0.0
    solves = 0.0
    for j in range(n):
        km = min(b, n - 1 - j)
        lu += km + 2.0 * km * km
        solves += 2.0 * km + 1.0 + 2.0 * min(b, j)
    return lu + 60.0 * solves


def leaf_solve_flops_per_rhs() -> float:
    """FP64 FLOPs of one leaf solve sweep pair for one right-hand side: L (bandwidth 15) and
    U (bandwidth 15, reciprocal pivots)."""
    n, b = 225, 15
    return sum(2.0 * min(b, n - 1 - j) + 1.0 + 2.0 * min(b, j) for j in range(n))


def peaks() -> dict:
    p = {"hbm_gbs": None, "bf16_tflops": None}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        p.update({k: m.get(k) for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained", "sm_max_mhz")})
    except OSError:
        pass
    return p


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: str):
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "-i", gpu,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.out.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(pg, x: float) -> float:
    """The largest x over all ranks (every rank gets it); x itself without a process group."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t[0])


def job_value(ws: int, steps: int, n: int, seconds: float) -> float:
    """Whole-job throughput in DOF/s: every one of ws ranks solved steps problems of n unknowns
    (weak scaling), and the slowest rank took seconds."""
    return ws * steps * n / seconds


# ------------------------------------------------------------------ CPU oracle leg
def oracle_sample(n: int, nrhs: int, seed: int = 1):
    """Factor + solve + GMRES refinement of one instance with the CPU oracle; returns
    (DOF/s, seconds, relres max, cores used)."""
    import numpy as np

    import workloads as W
    from oracle.gmres import gmres
    from oracle.nd import nested_dissection
    from oracle.spalu import Options, factor, solve
    P = W.make_problem("diffusion", n, seed=seed, nrhs=nrhs)
    nd = nested_dissection(n, n)
    t0 = time.perf_counter()
    F = factor(P.A, nd, Options(eps=EPS_ID, symmetric=True))
    X = solve(F, P.B)
    rel = []
    for c in range(nrhs):
        x, _, r = gmres(P.A.matvec, lambda v: solve(F, v), P.B[:, c], X[:, c], m=30, tol=1e-10)
        X[:, c] = x
        rel.append(r)
    t = time.perf_counter() - t0
    return n * n / t, t, max(rel), 1


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = args.ref_n
    times = []
    for i in range(args.warmup + args.steps):
        _, t, rel, cores = oracle_sample(n, NRHS, seed=1 + i)
        if i >= args.warmup:
            times.append(t)
    tot = sum(times)
    value = args.steps * n * n / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"diffusion {n}x{n} a=exp(GRF l=0.05 var=1), {NRHS} normal RHS, "
                               f"eps_ID={EPS_ID}, GMRES to 1e-10 (bounded sample of the "
                               f"{N_SIDE}x{N_SIDE} workload)", "N": n * n, "nrhs": NRHS},
        "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n}x{n} instance of the same problem family, {NRHS} RHS, "
                                   "factor + solve + GMRES per step"},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU leg
def _leaf_flops_split():
    """(FP64 FLOPs of the band LU, FLOPs of the 60 band solves) of one leaf elimination."""
    n, b = 225, 15
    lu = sum(min(b, n - 1 - j) + 2.0 * min(b, n - 1 - j) ** 2 for j in range(n))
    return lu, leaf_algorithmic_flops() - lu


def measured_alu_peaks() -> dict:
    """FP64 and FP32 FMA rates of this GPU's CUDA cores, measured by the library's probe
    kernel (FLOP/s); the unit-count figures (152 SMs x 4 / 256 FLOP per clock x 2070 MHz)
    only where the probe cannot run."""
    try:
        from paper_2408_14193_gb300.spalu import measure_fma_peak
        return {"fp64": measure_fma_peak(0), "fp32": measure_fma_peak(1), "source": "measured (FMA probe kernel)"}
    except Exception as exc:                 # noqa: BLE001
        clk = SM_MAX_MHZ * 1e6
        return {"fp64": N_SM * FP64_FLOP_PER_CLK_SM * clk, "fp32": N_SM * FP32_FLOP_PER_CLK_SM * clk,
                "source": f"derived from unit counts ({exc})"}


def _sum_levels(st, key):
    return float(sum(lv.get(key, 0) for lv in st["levels"]))


def _roofline(st, steps, fp32: bool, hbm_gbs: float, alu: dict):
    """Roofline of the dominant kernel of the step: the sparsification (sparsify_kernel, all
    levels; its launches carry the ID, the transforms and the remainder eliminations).
    achieved = the algorithmic FLOPs its launches counted (per level: sketch 2 h |F| e,
    pivoted QR, interpolation, transforms, remainder eliminations; work.cuh) / their CUDA-event
    time inside the timed steps; peak = the measured FMA rate of the precision its arithmetic
    runs in (FP32 in the mixed path, FP64 otherwise)."""
    tms, tcount = st["timing_ms"], st["timing_count"]
    sp_ms = sum(v for k, v in tms.items() if k.startswith("sparsify_l"))
    launches = sum(v for k, v in tcount.items() if k.startswith("sparsify_l"))
    flops = _sum_levels(st, "flops_sparsify")          # per factorization = per step
    peak = alu["fp32" if fp32 else "fp64"]
    ach = flops / (sp_ms / steps / 1e3)
    per_level = []
    for lv in st["levels"]:
        t = tms.get(f"sparsify_l{lv['level']}", 0.0) / steps
        if t > 0:
            per_level.append({"level": lv["level"], "ms": round(t, 4), "gflop": round(lv["flops_sparsify"] / 1e9, 4),
                              "tflops": round(lv["flops_sparsify"] / (t / 1e3) / 1e12, 4)})
    return {"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": None, "kernel": "sparsify_kernel (all levels)",
            "algorithmic_flops": flops, "launches_per_step": launches / steps,
            "launch_ms": sp_ms / launches if launches else None, "share_of_step_ms": sp_ms / steps,
            "peak_source": f"{alu['source']}, {'FP32' if fp32 else 'FP64'} CUDA cores",
            "per_level": per_level}


def _step_roofline(st, steps, ms_per_step: float, fp32: bool, nrhs: int, n_solves: int, gmres_iters: int,
                   hbm_gbs: float, alu: dict):
    """Whole-step roofline: T_roof = sum over phases of max(FP64 FLOPs / P64 + FP32 FLOPs /
    P32, bytes / HBM), against the measured step time.  Work per phase:
      leaf elimination   band LU (FP64) + 60 band solves per leaf (FP32 in the mixed path);
      sparsify, merge    the counted algorithmic FLOPs (precision of the path);
      each solve         bytes: the leaf factors (band L/U, pivots; the mixed path's backward
                         step reads the 225 x 60 operator), the segment and separator factors
                         twice (forward, backward), and the solve vector read and written per
                         sweep (leaf sweeps, the 2 level sweeps);
      GMRES              per iteration: SpMV (5 FMA per row and column) and modified
                         Gram-Schmidt against j + 1 basis vectors (2 FMA each), FP64."""
    N = N_SIDE * N_SIDE
    nleaf = ((N_SIDE + 1) // 16) ** 2
    p64, p32 = alu["fp64"], alu["fp32"]
    pa = p32 if fp32 else p64
    hb = hbm_gbs * 1e9
    tb = 4 if fp32 else 8
    lu, sv = _leaf_flops_split()
    phases = {}
    phases["leaf_factor"] = nleaf * (lu / p64 + sv / pa)
    phases["sparsify"] = _sum_levels(st, "flops_sparsify") / pa
    phases["merge"] = _sum_levels(st, "flops_merge") / pa
    tape = _sum_levels(st, "bytes_seg") + _sum_levels(st, "bytes_sep")
    leaf_f = nleaf * (225 * 31 * tb + 225 * 4)
    leaf_b = nleaf * 225 * 60 * 4 if fp32 else leaf_f
    vec = N * nrhs * tb
    solve_bytes = leaf_f + leaf_b + 2 * tape + 8 * vec
    phases["solves"] = n_solves * solve_bytes / hb
    g64 = 0.0
    for j in range(gmres_iters):
        g64 += N * nrhs * (10 + 4 * (j + 1))
    g64 += N * nrhs * 10                            # the residual of the initial guess
    phases["gmres"] = g64 / p64
    t_roof = sum(phases.values())
    return {"t_roof_ms": t_roof * 1e3, "t_measured_ms": ms_per_step, "frac": t_roof * 1e3 / ms_per_step,
            "phases_roof_ms": {k: round(v * 1e3, 4) for k, v in phases.items()},
            "solve_bytes": solve_bytes, "peaks": {"fp64_tflops": p64 / 1e12, "fp32_tflops": p32 / 1e12,
                                                  "hbm_gbs": hbm_gbs, "alu_source": alu["source"]}}


def _nvtx(push: bool):
    try:
        import torch
        if push:
            torch.cuda.nvtx.range_push("step")
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def train_predictor(dev, prec, eps, epochs: int = 200):
    """Record adaptive-ID rows on TRAIN_SET (same precision and eps as the timed path), fit
    the standardisation and train the network on the GPU; returns (predictor, info)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2408_14193_gb300 import Factor, NestedDissection, Predictor
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xs, Ys = [], []
    for kind, n, seed in TRAIN_SET:
        P = W.make_problem(kind, n, seed=seed, nrhs=1)
        f = Factor(NestedDissection(n), eps_id=eps, symmetric=1 if P.symmetric else 0, precision=prec)
        f.set_predictor(None, "record")
        f.factor(torch.from_numpy(P.A.indptr).to(dev), torch.from_numpy(P.A.indices).to(dev),
                 torch.from_numpy(P.A.data).to(dev))
        X, Y = f.export_training()
        Xs.append(X)
        Ys.append(Y)
    X = torch.cat(Xs).contiguous()
    Y = torch.cat(Ys).contiguous()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    p = Predictor(W.predictor_init_params(0))
    p.fit_norm(X)
    loss0, _ = p.loss_grad(X, Y)
    loss = p.train(X, Y, epochs=epochs, batch=256, lr=3e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return p, {"rows": int(X.shape[0]), "record_s": round(t1 - t0, 3), "train_s": round(t2 - t1, 3),
               "epochs": epochs, "batch": 256, "loss_initial": loss0, "loss_final": loss,
               "problems": [f"{k} {n}x{n}" for k, n, _ in TRAIN_SET]}


def run_batch(args, emit: bool = True):
    """Batched factorization + solve + refinement of 256 independent variable-coefficient
    diffusion problems (config 4 shape): side lengths drawn from {63, 127, 255, 511}, each with
    its own a = exp(GRF) field and one standard-normal right-hand side (seeded), mixed precision
    at the mixed eps_ID, refined by GMRES to 1e-10.  All problems' factorizations, solves and GMRES
    cycles are one CUDA graph (spalu_batch_graph_*, 16 concurrent branches); the same work
    through the plain calls (batched factorization on 16 streams, then solve and refinement
    per problem) is timed beside it.  Aggregate DOF/s = total unknowns / time per batch."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    import workloads as W
    ge.build()
    from paper_2408_14193_gb300 import BatchGraph, Factor, NestedDissection, factor_batch
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(4)
    nprob = args.batch_n
    sizes = rng.choice([63, 127, 255, 511], size=nprob)
    nds = {int(n): NestedDissection(int(n)) for n in set(sizes.tolist())}
    t0 = time.perf_counter()
    probs = []
    for i, n in enumerate(sizes.tolist()):
        P = W.make_problem("diffusion", n, seed=4000 + i, nrhs=1)
        csr = (torch.from_numpy(P.A.indptr).to(dev), torch.from_numpy(P.A.indices).to(dev),
               torch.from_numpy(P.A.data).to(dev))
        probs.append((n, P, csr, torch.from_numpy(np.ascontiguousarray(P.B.T)).to(dev)))
    gen_s = time.perf_counter() - t0
    eps = args.mixed_eps
    fs = [Factor(nds[n], eps_id=eps, symmetric=1, precision=1) for n, _, _, _ in probs]
    Xs = [torch.zeros_like(B) for _, _, _, B in probs]
    t0 = time.perf_counter()
    bg = BatchGraph(fs, [c for _, _, c, _ in probs], [B for _, _, _, B in probs], Xs, nstreams=16)
    torch.cuda.synchronize()
    cap_s = time.perf_counter() - t0
    dofs = int(sum(n * n for n, _, _, _ in probs))
    stream = torch.cuda.current_stream()

    def timed(step, k):
        ms = 0.0
        out = None
        for _ in range(k):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = step()
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        return ms / k, out

    for _ in range(args.warmup):
        bg.run()
    torch.cuda.synchronize()
    ms_graph, (its, rel) = timed(bg.run, args.steps)
    # the same work through the plain calls
    gs = [Factor(nds[n], eps_id=eps, symmetric=1, precision=1) for n, _, _, _ in probs]
    streams = [torch.cuda.Stream() for _ in range(16)]

    def plain():
        factor_batch(gs, [c for _, _, c, _ in probs], [streams[i % 16] for i in range(nprob)])
        r = []
        for g, (_, _, _, B), X in zip(gs, probs, Xs):
            g.solve(B, X)
            r.append(float(np.max(g.refine(B, X)[1])))
        return r

    for _ in range(args.warmup):
        plain()
    torch.cuda.synchronize()
    ms_plain, rel_plain = timed(plain, max(1, args.steps // 2))
    # CPU residual of a sample of the graph's solutions
    res = []
    bg.run()
    torch.cuda.synchronize()
    for i in range(0, nprob, max(1, nprob // 16)):
        n, P, _, _ = probs[i]
        x = Xs[i].cpu().numpy().T
        res.append(float(np.max(np.linalg.norm(P.B - P.A.matvec(x), axis=0) / np.linalg.norm(P.B, axis=0))))
    line = {"metric": "aggregate factor+solve DOF/s, 256 independent diffusion problems (batched)",
            "value": dofs / (ms_graph / 1e3), "unit": "DOF/s", "ms_per_batch": ms_graph, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"{nprob} diffusion problems, sides from {{63,127,255,511}} (seed 4), each its "
                                   f"own a=exp(GRF l=0.05 var=1) field (seed 4000+i), 1 normal RHS each, mixed "
                                   f"precision, eps_ID={eps}, GMRES to 1e-10; one CUDA graph over all problems "
                                   f"(16 branches)",
                       "problems": nprob, "dofs": dofs, "branches": 16,
                       "sizes": {str(k): int((sizes == k).sum()) for k in sorted(nds)}},
            "gmres_iters_max": int(np.max(its)), "relres_max": float(np.max(rel)),
            "relres_cpu_sample_max": max(res),
            "plain_calls": {"value": dofs / (ms_plain / 1e3), "ms_per_batch": ms_plain,
                            "relres_max": max(rel_plain),
                            "what": "spalu_factor_numeric_batch on 16 streams, then spalu_solve + spalu_refine "
                                    "per problem"},
            "generate_s": round(gen_s, 1), "create_and_capture_s": round(cap_s, 1)}
    if emit:
        print(json.dumps(line), flush=True)
    del bg, fs, gs
    torch.cuda.empty_cache()
    return line


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__ as ge
    import workloads as W
    ws, rank, local = dist_env()
    torch.cuda.set_device(local if torch.cuda.device_count() > local else 0)
    dev = torch.device("cuda", torch.cuda.current_device())
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    ge.build()
    from paper_2408_14193_gb300 import Factor, NestedDissection
    from paper_2408_14193_gb300.spalu import kernel_launches

    P = W.make_problem("diffusion", N_SIDE, seed=1 + rank, nrhs=NRHS)
    N = P.A.n
    A = P.A
    rp = torch.from_numpy(A.indptr).to(dev)
    ci = torch.from_numpy(A.indices).to(dev)
    va = torch.from_numpy(A.data).to(dev)
    B = torch.from_numpy(np.ascontiguousarray(P.B.T)).to(dev)
    X = torch.empty_like(B)
    t_nd = time.perf_counter()
    nd = NestedDissection(N_SIDE)
    torch.cuda.synchronize()
    nd_s = time.perf_counter() - t_nd
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", "") or "")
    gpu_id = ("GPU-" + gpu_id) if gpu_id and not gpu_id.startswith("GPU-") else (gpu_id or str(local))

    def measure(prec, eps, sample_clocks, pred=None, graph=not args.no_graph, near_radius=2, prob=None,
                steps=None, tune=True, schur_tc=1, sketch_tc=0):
        pnd, prp, pci, pva, pB, pX, psym = prob or (nd, rp, ci, va, B, X, 1)
        nsteps = steps or args.steps
        f = Factor(pnd, eps_id=eps, symmetric=psym, precision=prec, near_radius=near_radius, schur_tc=schur_tc,
                   sketch_tc=sketch_tc)
        if pred is not None:
            f.set_predictor(pred, "predict", margin=PRED_MARGIN)

        def step():
            if graph:                             # factor + solve + refine as one CUDA graph
                return f.factor_solve_graph(prp, pci, pva, pB, pX)
            f.factor(prp, pci, pva)
            f.solve(pB, pX)
            return f.refine(pB, pX)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if tune:
            f.tune_factor()                       # sparsify occupancy per level (untimed)
            f.tune_solve(min(16, int(pB.shape[0])))   # CTA widths of the level solves (untimed)
        f.set_timing(True)                        # phase events (captured into the graph too)
        step()                                    # plain run + capture after the tuners
        step()
        torch.cuda.synchronize()
        f.set_timing(True)                        # resets the sums
        sampler = ClockSampler(gpu_id) if sample_clocks else None
        time.sleep(0.3)
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        l0 = kernel_launches()
        ms = 0.0
        iters, rels = [], []
        for _ in range(nsteps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            _nvtx(True)                           # the timed kernels (for profiler filters)
            e0.record(stream)
            it, rel = step()
            e1.record(stream)
            _nvtx(False)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            iters.append(it)
            rels.append(float(np.max(rel)))
        torch.cuda.synchronize()
        launches = kernel_launches() - l0
        if pg:
            pg.barrier()
        clocks = sampler.stop() if sampler else None
        st = f.stats()
        f.set_timing(False)
        del f
        ms = max_over_ranks(pg, ms)
        return {"ms": ms, "iters": max(iters), "relres": max(rels), "launches": launches,
                "st": st, "clocks": clocks,
                "sparsify_ms_per_level": {str(lv["level"]): round(st["timing_ms"].get(f"sparsify_l{lv['level']}", 0.0)
                                                                 / nsteps, 4) for lv in st["levels"]},
                "merge_ms": sum(v for k, v in st["timing_ms"].items() if k.startswith("merge_l")) / nsteps}

    def other_config(kind, n, nrhs, prec, eps, sym, steps, tune, pred=None):
        """One more workload of the configuration list (its own generated problem)."""
        Q = W.make_problem(kind, n, seed=2 + rank, nrhs=nrhs)
        qd = (NestedDissection(n), torch.from_numpy(Q.A.indptr).to(dev), torch.from_numpy(Q.A.indices).to(dev),
              torch.from_numpy(Q.A.data).to(dev))
        QB = torch.from_numpy(np.ascontiguousarray(Q.B.T)).to(dev)
        r = measure(prec, eps, False, pred=pred, prob=qd + (QB, torch.zeros_like(QB), sym), steps=steps, tune=tune)
        out = {"value": job_value(ws, steps, n * n, r["ms"] / 1e3), "unit": "DOF/s", "ms_per_step": r["ms"] / steps,
               "N": n * n, "nrhs": nrhs, "precision": "mixed" if prec else "fp64", "eps_id": eps,
               "relres_max": r["relres"], "gmres_iters": r["iters"], "steps": steps,
               "k_max": max(lv["k_max"] for lv in r["st"]["levels"]),
               "e_max": max(lv["e_max"] for lv in r["st"]["levels"])}
        del qd, QB
        torch.cuda.empty_cache()
        return out

    alu = measured_alu_peaks()
    pred, pred_info = train_predictor(dev, 1, args.mixed_eps, args.pred_epochs)
    if args.factor_only:
        # profiling runs: the headline matrix factored (mixed precision, learned ranks) warmup +
        # steps times, nothing else on the device (no solve vectors, no GMRES basis)
        f = Factor(nd, eps_id=args.mixed_eps, symmetric=1, precision=1, schur_tc=1 if args.schur_tc else 0)
        f.set_predictor(pred, "predict", margin=PRED_MARGIN)
        for _ in range(args.warmup + args.steps):
            f.factor(rp, ci, va)
        torch.cuda.synchronize()
        print(json.dumps({"factorizations": args.warmup + args.steps,
                          "arena_bytes": f.stats()["arena_bytes"]}), flush=True)
        return 0
    head = measure(1, args.mixed_eps, True, pred)  # mixed precision + learned ranks: the headline
    if args.only_mixed:                           # profiling runs: the headline path alone
        print(json.dumps({"ms_per_step": head["ms"] / args.steps, "relres_max": head["relres"],
                          "gmres_iters": head["iters"],
                          "phase_ms_per_step": {k: round(v / args.steps, 4)
                                                for k, v in sorted(head["st"]["timing_ms"].items())}}), flush=True)
        return 0
    base = measure(0, EPS_ID, False)              # plain FP64 GPU form
    base_loose = measure(0, args.mixed_eps, False)   # FP64 at the mixed path's eps_ID
    noml = measure(1, args.mixed_eps, False)      # ablation: mixed precision, adaptive ID
    prnd = measure(1, args.mixed_eps, False, near_radius=-1)   # ablation: pure randomized sampling
    scc = measure(1, args.mixed_eps, False, schur_tc=0)      # ablation: Schur updates on the CUDA cores
    sktc = measure(1, args.mixed_eps, False, sketch_tc=1)    # ablation: sketch products on the tensor cores
    cfg3 = cfg2 = None
    if not args.no_configs:
        # convection-diffusion 1023^2, 4 RHS, learned predictor on (the non-symmetric family)
        cfg3 = dict(other_config("convdiff", N_SIDE, 4, 1, args.mixed_eps, 0, args.steps, True, pred),
                    workload=f"convection-diffusion {N_SIDE}x{N_SIDE}, beta=50(cos t, sin t), first-order upwind, "
                             "4 normal RHS, mixed precision, learned ranks, GMRES to 1e-10")
        # Helmholtz 2047^2 at 10 points per wavelength, 8 point sources: the FP32 factor of this
        # indefinite operator leaves GMRES without convergence, so the factor is FP64
        cfg2 = dict(other_config("helmholtz", 2047, 8, 0, EPS_ID, 1, 3, False),
                    workload="Helmholtz 2047x2047, k0 = 2 pi / (10 h), k^2 (1 + 0.2 GRF), 8 Gaussian point "
                             "sources, FP64 factor (the mixed one does not converge), eps_ID=1e-8, GMRES to 1e-10")

    # end to end through the host-memory entry points (pinned host buffers), headline path
    val_h = torch.from_numpy(A.data).pin_memory().numpy()
    rp_h = torch.from_numpy(A.indptr).pin_memory().numpy()
    ci_h = torch.from_numpy(A.indices).pin_memory().numpy()
    B_h = torch.from_numpy(np.ascontiguousarray(P.B.T)).pin_memory().numpy()
    X_h = torch.empty(tuple(B_h.shape), dtype=torch.float64).pin_memory().numpy()
    g = Factor(nd, eps_id=args.mixed_eps, symmetric=1, precision=1)
    g.set_predictor(pred, "predict", margin=PRED_MARGIN)
    g.factor_host(rp_h, ci_h, val_h)
    g.tune_factor()
    g.tune_solve(NRHS)
    g.factor_solve_host(rp_h, ci_h, val_h, B_h, refine=True, out=X_h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_rel = 0.0
    for _ in range(args.steps):
        Xh, _, rel = g.factor_solve_host(rp_h, ci_h, val_h, B_h, refine=True, out=X_h)
        e2e_rel = max(e2e_rel, float(np.max(rel)))
    e2e_s = time.perf_counter() - t0
    del g
    e2e_s = max_over_ranks(pg, e2e_s)
    if rank != 0:
        pg.destroy_process_group()
        return 0
    value = job_value(ws, args.steps, N, head["ms"] / 1e3)
    base_value = job_value(ws, args.steps, N, base["ms"] / 1e3)
    noml_value = job_value(ws, args.steps, N, noml["ms"] / 1e3)
    pk = peaks()
    hbm = pk.get("hbm_gbs") or 6800.0
    e2e_value = job_value(ws, args.steps, N, e2e_s)

    batch = None
    if ws == 1 and not args.no_batch:           # the batched workload, timed after the headline
        batch = run_batch(argparse.Namespace(**dict(vars(args), steps=3, warmup=1)), emit=False)
    cpu = None
    if ws == 1 and not args.no_cpu:
        v, t, rel, cores = oracle_sample(args.cpu_n, NRHS)
        cpu = {"value": v, "unit": "DOF/s", "cores": cores, "kind": "oracle",
               "sample": f"one {args.cpu_n}x{args.cpu_n} instance of the same family, {NRHS} RHS, "
                         f"factor + solve + GMRES to 1e-10 ({t:.1f} s)"}
    st = head["st"]
    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"diffusion {N_SIDE}x{N_SIDE} a=exp(GRF l=0.05 var=1), {NRHS} normal "
                               f"RHS, mixed precision (FP32 factors and solve, FP64 leaf LU and "
                               f"QR pivots/norms), eps_ID={args.mixed_eps}, GMRES (FP64 residual) "
                               f"to 1e-10",
                   "N": N, "nrhs": NRHS, "precision": "mixed", "eps_id": args.mixed_eps,
                   "learned_ranks": True, "step": "one CUDA graph (factor, solve, refine)" if not args.no_graph
                   else "plain calls (factor, solve, refine)",
                   "l2": "256 MB flush between steps; factor working set > L2"},
        "relres_max": head["relres"], "gmres_iters": head["iters"],
        "fp64_plain": {"value": base_value, "unit": "DOF/s", "ms_per_step": base["ms"] / args.steps,
                       "eps_id": EPS_ID, "relres_max": base["relres"], "gmres_iters": base["iters"],
                       "phase_ms_per_step": {k: round(v / args.steps, 4) for k, v in sorted(base["st"]["timing_ms"].items())},
                       "roofline": _roofline(base["st"], args.steps, False, hbm, alu)},
        "fp64_plain_same_eps": {"value": job_value(ws, args.steps, N, base_loose["ms"] / 1e3), "unit": "DOF/s",
                                "ms_per_step": base_loose["ms"] / args.steps, "eps_id": args.mixed_eps,
                                "relres_max": base_loose["relres"], "gmres_iters": base_loose["iters"]},
        "mixed_adaptive": {"value": noml_value, "unit": "DOF/s", "ms_per_step": noml["ms"] / args.steps,
                           "relres_max": noml["relres"], "gmres_iters": noml["iters"],
                           "id_passes": sum(lv["passes"] for lv in noml["st"]["levels"]),
                           "sparsify_ms_per_level": noml["sparsify_ms_per_level"]},
        "sampling_ablation": {"what": "mixed, adaptive ID, pure randomized sampling (every neighbour row "
                                      "sketched, Sec. 4.2.1) against the hybrid sampling of mixed_adaptive",
                              "value": job_value(ws, args.steps, N, prnd["ms"] / 1e3), "unit": "DOF/s",
                              "ms_per_step": prnd["ms"] / args.steps, "relres_max": prnd["relres"],
                              "gmres_iters": prnd["iters"],
                              "k_sum": sum(lv["k_sum"] for lv in prnd["st"]["levels"]),
                              "k_sum_hybrid": sum(lv["k_sum"] for lv in noml["st"]["levels"]),
                              "sparsify_gflop": sum(lv["flops_sparsify"] for lv in prnd["st"]["levels"]) / 1e9,
                              "sparsify_gflop_hybrid": sum(lv["flops_sparsify"] for lv in noml["st"]["levels"]) / 1e9,
                              "sparsify_ms_per_level": prnd["sparsify_ms_per_level"]},
        "schur_cuda_cores": {"what": "mixed, adaptive ID, separator Schur updates M -= Z W in FP32 on the CUDA "
                                     "cores, against the tensor-core updates (mma.sync TF32, operands split into "
                                     "high and low parts, 3 products) of mixed_adaptive and the headline",
                             "value": job_value(ws, args.steps, N, scc["ms"] / 1e3), "unit": "DOF/s",
                             "ms_per_step": scc["ms"] / args.steps, "gmres_iters": scc["iters"],
                             "relres_max": scc["relres"], "merge_ms_per_step": scc["merge_ms"],
                             "merge_ms_per_step_tensor_cores": noml["merge_ms"]},
        "sketch_tensor_cores": {"what": "mixed, adaptive ID, sketch products G B_F on the tensor cores (split-TF32 "
                                        "mma.sync) against the FP32 CUDA-core products of mixed_adaptive",
                                "value": job_value(ws, args.steps, N, sktc["ms"] / 1e3), "unit": "DOF/s",
                                "ms_per_step": sktc["ms"] / args.steps, "gmres_iters": sktc["iters"],
                                "relres_max": sktc["relres"],
                                "sparsify_ms_per_step": sum(sktc["sparsify_ms_per_level"].values()),
                                "sparsify_ms_per_step_cuda_cores": sum(noml["sparsify_ms_per_level"].values())},
        "predictor": dict(pred_info, margin=PRED_MARGIN, id_passes=sum(lv["passes"] for lv in st["levels"]),
                          predicted=sum(lv["predicted"] for lv in st["levels"]),
                          fallbacks=sum(lv["fallbacks"] for lv in st["levels"]),
                          levels_on=[lv["level"] for lv in st["levels"] if lv.get("predictor") == 2],
                          sparsify_ms_per_level=head["sparsify_ms_per_level"]),
        "speedup_vs_fp64": value / base_value,
        "nd_build_s": nd_s,
        "clocks": head["clocks"],
        "e2e": {"value": e2e_value, "unit": "DOF/s",
                "h2d_bytes_per_step": int(A.data.nbytes + A.indptr.nbytes + A.indices.nbytes + P.B.nbytes),
                "d2h_bytes_per_step": int(P.B.nbytes), "relres_max": e2e_rel},
        "gpu_launches": int(head["launches"]),
        "roofline": _roofline(st, args.steps, True, hbm, alu),
        "step_roofline": _step_roofline(st, args.steps, head["ms"] / args.steps, True, NRHS, 1 + head["iters"],
                                        head["iters"], hbm, alu),
        "phase_ms_per_step": {k: round(v / args.steps, 4) for k, v in sorted(st["timing_ms"].items())},
        "factor_stats": {"q_tilde": st["q_tilde"], "levels": st["levels"]},
        "step_graph": st.get("step_graph"),
        "cpu_baseline": cpu,
        "batch": batch,
        "config3_convdiff": cfg3,
        "config2_helmholtz": cfg2,
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-n", type=int, default=255, dest="cpu_n")
    ap.add_argument("--ref-n", type=int, default=127, dest="ref_n")
    ap.add_argument("--no-cpu", action="store_true", dest="no_cpu")
    # 4e-7: three GMRES iterations reach 1e-10 with a ~10x margin (1.1e-11 measured); at 5e-7
    # they land at 8e-11 .. 9e-11, and a retrained network that gives slightly smaller ranks
    # then needs a fourth (a fifth solve); at 1e-6 the fourth is the rule
    ap.add_argument("--mixed-eps", type=float, default=4e-7, dest="mixed_eps")
    ap.add_argument("--pred-epochs", type=int, default=200, dest="pred_epochs")
    ap.add_argument("--no-graph", action="store_true", dest="no_graph",
                    help="time the plain calls (factor, solve, refine) instead of the captured step graph")
    ap.add_argument("--schur-cuda-cores", action="store_false", dest="schur_tc",
                    help="with --factor-only: separator Schur updates on the CUDA cores")
    ap.add_argument("--factor-only", action="store_true", dest="factor_only",
                    help="factor the headline matrix warmup + steps times and exit (profiler runs)")
    ap.add_argument("--only-mixed", action="store_true", dest="only_mixed",
                    help="time the mixed-precision path only (for profiler runs)")
    ap.add_argument("--batch", action="store_true",
                    help="the batched workload (256 independent problems) instead of the headline")
    ap.add_argument("--batch-n", type=int, default=256, dest="batch_n")
    ap.add_argument("--no-configs", action="store_true", dest="no_configs",
                    help="leave the convection-diffusion and Helmholtz workloads out of the headline run")
    ap.add_argument("--no-batch", action="store_true", dest="no_batch",
                    help="leave the batched workload out of the headline run")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batch:
        run_batch(args)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
