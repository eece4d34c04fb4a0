"""Host logic of bench.py on the CPU.  Multi-rank, world size 2: the max-over-ranks timing
reduction over gloo (each rank its own spawned process, rendezvous on 127.0.0.1, as under
torchrun), the whole-job (weak-scaling) throughput, and the reference arm's rule that rank 0
alone runs and prints.  Measurement: the roofline arithmetic of the bench line (the
sparsification against the measured FMA peak, the whole-step roofline).  No GPU is touched."""
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


def test_roofline_arithmetic():
    """The bench line's roofline of the sparsification from synthetic timings and counters:
    achieved = counted algorithmic FLOPs per step / sparsify time per step, frac = achieved /
    measured FMA peak of the path's precision; the whole-step roofline adds up its phases."""
    sys.path.insert(0, ROOT)
    import bench
    steps = 5
    st = {"timing_ms": {"leaf_factor": 5 * 1.6, "sparsify_l12": 5 * 2.0, "sparsify_l11": 5 * 1.5},
          "timing_count": {"leaf_factor": 5, "sparsify_l12": 5, "sparsify_l11": 5},
          "levels": [{"level": 11, "flops_sparsify": 3e9, "flops_merge": 1e8, "bytes_seg": 2e7, "bytes_sep": 4e6},
                     {"level": 12, "flops_sparsify": 4e9, "flops_merge": 2e8, "bytes_seg": 3e7, "bytes_sep": 5e6}]}
    alu = {"fp64": 1.2e12, "fp32": 75e12, "source": "synthetic"}
    r = bench._roofline(st, steps, True, 6800.0, alu)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["algorithmic_flops"] == pytest.approx(7e9)
    assert r["achieved"] == pytest.approx(7e9 / 3.5e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 75.0)
    assert r["launch_ms"] == pytest.approx(3.5 / 2) and r["share_of_step_ms"] == pytest.approx(3.5)
    assert [p["level"] for p in r["per_level"]] == [11, 12]
    r64 = bench._roofline(st, steps, False, 6800.0, alu)
    assert r64["peak"] == pytest.approx(1.2) and r64["frac"] == pytest.approx(r64["achieved"] / 1.2)
    sr = bench._step_roofline(st, steps, 18.0, True, 16, 4, 3, 6800.0, alu)
    assert sr["t_roof_ms"] == pytest.approx(sum(sr["phases_roof_ms"].values()), rel=1e-3)
    assert sr["phases_roof_ms"]["sparsify"] == pytest.approx(7e9 / 75e12 * 1e3, rel=1e-3)
    assert 0 < sr["frac"] < 1 and sr["frac"] == pytest.approx(sr["t_roof_ms"] / 18.0)
