"""The multi-rank host logic of bench.py on the CPU (gloo, world size 2).

Under torchrun every rank trains its own replica of the workload with no
collective on the data path; the only cross-rank steps are the barriers around
the timed region and the max over ranks of the measured time, from which the
whole-job throughput follows.  Those run here as two gloo processes; the
reference arm's other ranks must exit 0 without work."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    try:
        dist.barrier()
        local_ms = 10.0 + 5.0 * rank            # rank 1 is the slower replica
        job_ms = bench.max_over_ranks(local_ms, 2, "cpu")
        value = bench.job_throughput(2, 7, 1000, job_ms / 1e3)
        dist.barrier()
        q.put((rank, local_ms, job_ms, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert [g[0] for g in got] == [0, 1]
    for rank, local_ms, job_ms, value in got:
        assert job_ms == 15.0                   # both ranks see the slower rank's time
        assert value == pytest.approx(2 * 7 * 1000 / 0.015)   # units of both replicas / job time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput(1, 10, 100, 2.0) == 500.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1", MASTER_PORT="29599")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2",
                        "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
