"""The N > 1 replica path of bench.py on CPU: two gloo ranks, no GPU.

Each rank times its own shot; the job's value is the units all ranks processed over the
slowest rank's seconds, and the reference arm runs on rank 0 only.
"""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    # rank r: (r + 1) * 100 units in 0.5 + r seconds
    rate, sec = bench.job_rate(0.5 + rank, 100.0 * (rank + 1), ws, device="cpu")
    out.put((rank, rate, sec))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, rate, sec in res:
        assert sec == pytest.approx(1.5)            # the slowest rank
        assert rate == pytest.approx(300.0 / 1.5)   # units of both ranks


def test_job_rate_single_rank_is_plain_ratio():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(2.0, 10.0, 1) == (5.0, 2.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
