"""The benchmark's multi-rank contract on CPU ranks (gloo, world size 2):
every rank gets the slowest rank's time, the whole-job rate counts the units
of all ranks, and the reference arm runs on rank 0 only (the others exit 0
without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
# rank r took 10 + 7 r ms for its K = 50 steps
mx = bench.max_over_ranks(10.0 + 7.0 * rank, dist, "cpu")
rate = bench.whole_job_rate(world, 50, mx / 1e3)
dist.barrier()
print(json.dumps({"rank": rank, "max": mx, "rate": rate}), flush=True)
dist.destroy_process_group()
"""


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   BENCH_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["max"] == 17.0
        # 2 ranks x 50 steps in the slowest rank's 17 ms
        assert o["rate"] == pytest.approx(100 / 0.017)


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1, 10, 2.0) == 5.0


def test_reference_arm_rank0_only_under_torchrun():
    """`bench.py --impl reference` launched like the multi-GPU bench: one JSON
    line from rank 0, rank 1 exits 0 and prints nothing."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--workload", "blobs-2k",
           "--cpu-sample", "400"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    ln = lines[0]
    assert ln["impl"] == "reference" and ln["n_gpus"] == 2
    assert ln["value"] > 0 and ln["unit"] == "iter/s"
    assert ln["cpu_baseline"]["kind"] == "oracle" and ln["cpu_baseline"]["value"] == ln["value"]
    assert ln["e2e"]["h2d_bytes_per_step"] == 0 and ln["e2e"]["value"] == ln["value"]
    # the config names the sample that was timed; the full-N rate is a labelled extra
    assert ln["config"]["N"] <= ln["config"]["sample_of_N"] == 2000
    assert ln["cpu_baseline"]["cores"] >= 1
    ex = ln["extrapolated_to_full_N"]
    assert ex["N"] == 2000 and ex["value"] == pytest.approx(ln["value"] * ln["config"]["N"] / 2000, rel=1e-3)


def test_bench_args_and_bytes():
    import bench
    a = bench.parse_args(["--workload", "lowrank-2m", "--alpha", "0.5"])
    assert a.workload == "lowrank-2m" and a.alpha == 0.5 and a.mode == "bench"
    a = bench.parse_args(["--mode", "timing", "--sizes", "1000,2000", "--iters", "30"])
    assert a.mode == "timing" and a.sizes == "1000,2000" and a.iters == 30
    per = bench.algorithmic_bytes_per_point(50, 16, 32, 32, 32, 200)
    # the survey's per-point rule at the 1M-point workload: 33 FP32 rows of
    # D = 50 and the HD lists in the HD refinement; 64 gathered and 32
    # scattered LD rows (6,144 bytes) in the forces
    assert per["hd_refine"] == 33 * 200 + 8 * 32 + 8 * 32 + 4 * 32
    assert per["forces"] == 6144 and per["ld_refine"] == 33 * 64 + 8 * 32
    assert per["update"] == 6 * 64
    full = bench.full_bytes_per_point(50, 16, 32, 32, 32, 200)
    assert full["hd_refine"] == 33 * 200 + 8 * 32 + 4 * 32 + 80 + 8 * 32
    assert full["update"] == 7 * 64 and all(full[k] >= per[k] for k in per)
    assert bench.row_bytes_of(50) == {"fp32": 200, "bf16": 104, "fp8": 58}
