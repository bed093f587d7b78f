"""The N > 1 path of bench.py on CPU (gloo, world size 2): one replica per
rank, the job's time is the slowest rank's, the job's throughput counts every
rank's units, and under torchrun only rank 0 prints (the reference arm)."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import bench  # noqa: E402
import dist_helpers  # noqa: E402


def free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_single_process_helpers():
    assert bench.max_over_ranks(4.5, None, "cpu") == 4.5
    assert bench.job_rate(100.0, 1, 2.0) == 50.0
    assert bench.job_rate(100.0, 4, 2.0) == 200.0


def test_record_horizon_of_cycle_blocks():
    """The bench's horizon for streamed patches: how many cycles back a
    detector reads a record.  The surface and [[144,12,12]] memories compare
    consecutive rounds; the adaptive code's outer checks run every d/2 cycles
    (two at outer distance 4)."""
    from paper_2604_16613_gb300 import circuits as C
    nm = C.NoiseModel.uniform(1e-3)
    assert bench.record_horizon(C.rotated_surface_code_memory(5, 5, nm).cycle_blocks()) == 1
    assert bench.record_horizon(C.bb_memory(3, nm, seed=3).cycle_blocks()) == 1
    ad = C.concatenated_adaptive_branch(4, 9, seed=5, noise=nm, layout=C.ConcatenatedLayout(4))
    assert bench.record_horizon(ad.cycle_blocks()) == 2


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=dist_helpers.max_over_ranks_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(queue.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, (r, slowest, rate, env) in enumerate(out):
        assert r == rank
        assert slowest == 13.0                  # both ranks see the slower one
        assert rate == pytest.approx(2 * 1000.0 / 13.0)
        assert env == (2, rank, rank)


def test_reference_arm_under_torchrun_world2():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1                      # rank 0 alone prints
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle"
