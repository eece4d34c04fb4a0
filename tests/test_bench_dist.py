"""Host logic of bench.py on the CPU.  Multi-rank, world size 2: the max-over-ranks timing
reduction over gloo (each rank its own spawned process, rendezvous on 127.0.0.1, as under
torchrun), the whole-job (weak-scaling) throughput, and the reference arm's rule that rank 0
alone runs and prints.  Measurement: the roofline and dominant-kernel arithmetic of the bench
line.  No GPU is touched."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, outdir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got = bench.max_over_ranks(dist, 10.0 * (rank + 1))     # rank r reports 10 (r + 1)
        dist.barrier()
        with open(os.path.join(outdir, f"rank{rank}.txt"), "w") as fh:
            fh.write(repr(got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_over_gloo(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    for r in range(ws):
        assert float((tmp_path / f"rank{r}.txt").read_text()) == 20.0   # every rank: the max


def test_max_over_ranks_without_a_group_and_job_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.5) == 3.5
    # weak scaling: two ranks that each solve 5 problems of 100 unknowns, the slower in 2 s
    assert bench.job_value(2, 5, 100, 2.0) == 500.0
    assert bench.job_value(2, 5, 100, 2.0) == 2 * bench.job_value(1, 5, 100, 2.0)


def _reference_arm(rank: int, ws: int):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0", "--ref-n", "31"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_runs_on_rank0_only():
    other = _reference_arm(1, 2)
    assert other.returncode == 0 and other.stdout.strip() == ""
    first = _reference_arm(0, 2)
    assert first.returncode == 0, first.stderr
    lines = [ln for ln in first.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["e2e"]["h2d_bytes_per_step"] == 0


def test_roofline_and_dominant_arithmetic():
    """The bench line's roofline and dominant-kernel entries from synthetic phase timings:
    the largest timed phase among those with a roof is chosen, achieved = algorithmic work /
    average launch time, frac = achieved / peak; the dominant entry is the sparsification's
    share of the step."""
    sys.path.insert(0, ROOT)
    import bench
    steps = 5
    st = {"timing_ms": {"leaf_factor": 5 * 1.6, "leaf_solve_fwd": 20 * 0.25, "leaf_solve_bwd": 20 * 0.14,
                        "sparsify_l12": 5 * 2.0, "sparsify_l11": 5 * 1.5},
          "timing_count": {"leaf_factor": 5, "leaf_solve_fwd": 20, "leaf_solve_bwd": 20,
                           "sparsify_l12": 5, "sparsify_l11": 5}}
    r = bench._roofline(st, steps, True, 6800.0)
    assert r["kernel"] == "leaf_lu_kernel+leaf_schur_kernel" and r["bound"] == "alu"
    assert r["launch_ms"] == pytest.approx(1.6) and r["share_of_step_ms"] == pytest.approx(1.6)
    assert r["achieved"] == pytest.approx(r["algorithmic_flops"] / 1.6e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"]) and 0 < r["frac"] < 1
    # with the leaf elimination faster, the forward sweeps (HBM-bound) are the largest phase
    st2 = {"timing_ms": dict(st["timing_ms"], leaf_factor=5 * 0.5), "timing_count": st["timing_count"]}
    r2 = bench._roofline(st2, steps, True, 6800.0)
    assert r2["kernel"] == "leaf_solve_kernel" and r2["unit"] == "GB/s" and r2["peak"] == 6800.0
    assert r2["achieved"] == pytest.approx(r2["algorithmic_bytes"] / 0.25e-3 / 1e9)
    dmn = bench._dominant(st, steps, 18.0)
    assert dmn["ms_per_step"] == pytest.approx(3.5) and dmn["share_of_step"] == pytest.approx(3.5 / 18.0)
    assert dmn["bound"] == "latency"
