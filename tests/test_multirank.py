"""The multi-process path of bench.py, on CPU with the gloo backend.

The solve does not shard: on N GPUs bench.py runs N independent solves, one per rank,
and the only collective is the reduction of the per-rank step times to the slowest one.
Two gloo ranks check that reduction and the whole-job rate, and that the reference arm
runs on rank 0 alone while the other ranks exit without work.
"""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))
    q.put((rank, ms, bench.job_value(world, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    assert [o[1] for o in out] == [15.0, 15.0]
    for _, ms, value in out:
        assert abs(value - 2 * 1e3 / 15.0) < 1e-12


def test_single_process_time_and_value():
    import bench
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.job_value(1, 250.0) == 4.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
