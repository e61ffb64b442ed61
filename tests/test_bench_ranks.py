"""The multi-process host logic of bench.py on CPU: two gloo ranks (one process
each, rendezvous on 127.0.0.1) take the slowest rank's time and the whole-job
throughput the way the GPU run does, and the reference arm works on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 1000.0 + 250.0 * rank  # rank 1 is the slower one
    total = bench.max_over_ranks(local_ms, world)
    out[rank] = (total, bench.job_value(world, 5, 30, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_the_whole_job_value():
    world, port = 2, _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        total, value = out[r]
        assert total == 1250.0
        assert value == pytest.approx(2 * 5 * 30 / 1.25)


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    """Under torchrun the non-zero ranks of --impl reference exit 0 without work."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_class_byte_models_count_the_basis_sizes_of_a_solve():
    """The roofline's algorithmic bytes per timing class, for a solve of 30 outer
    iterations (Solve-OF on iterations 1..29) with 20 GKS iterations from a 10-vector
    Golub-Kahan start: K = 10 + it vectors at GKS iteration it, so the projection pass with
    its Laplacian pass and append streams sum_{it<19} (19 + it) = 532 vectors per pair and
    call, s = V z sum_{it<20} (11 + it) = 410, the start's Gram columns
    sum_{j<10} (j + 1) = 55 plus 3 fields per column."""
    class W:
        nx, ny, nt = 16, 8, 5
    ns, P, calls = 16 * 8, 4, 29
    N2 = 2 * ns
    assert bench.class_bytes("of_subdot", W)[0] == calls * P * 4 * N2 * 532
    assert bench.class_bytes("of_combine", W)[0] == calls * P * 4 * N2 * 410
    assert bench.class_bytes("of_gram", W)[0] == calls * P * 4 * (N2 * 55 + 3 * ns * 10)
    assert bench.class_bytes("of_reorth", W) is None
    n = ns * 5
    assert bench.class_bytes("theta_gram", W)[0] == sum(4 * n * (10 + k) + 4 * n + 16 * P * ns for k in range(30))
    assert bench.class_bytes("small_solve", W) is None
    # with Solve-OF every 20 outer iterations (tau = 20) only k = 20 runs it
    assert bench.class_bytes("of_subdot", W, tau=20)[0] == 1 * P * 4 * N2 * 532
