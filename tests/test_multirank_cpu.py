"""The N > 1 path on CPU: world-size-2 gloo ranks run the bench's whole-job
rate (max elapsed over ranks, units of all ranks), the reference arm
leaves ranks other than 0 without work, and a rank that leaves between steps
makes the survivor's next collective fail instead of hang. Channels, sources
and streams are independent, so ranks are replicas: no data-path collective
exists to test."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    try:
        elapsed = [120.0, 150.0][rank]            # rank 1 is the slowest
        ms, value = bench.job_rate(elapsed, 1000.0, ws, steps=3, device="cpu")
        dist.barrier()
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_and_all_units():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, value in got:
        assert ms == 150.0
        assert value == pytest.approx(1000.0 * 2 * 3 / 0.150)


def test_job_rate_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.job_rate(200.0, 500.0, 1, steps=4, device="cpu")
    assert ms == 200.0 and value == pytest.approx(500.0 * 4 / 0.2)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def _rank_leaves(rank, ws, port, q):
    import datetime
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws, timeout=datetime.timedelta(seconds=10))
    dist.barrier()                                  # both ranks up
    if rank == 1:
        os._exit(3)                                 # leaves between steps, nothing in flight
    try:
        bench.job_rate(100.0, 1000.0, ws, steps=3, device="cpu")
        q.put((rank, "no error"))
    except Exception as e:                          # the collective ends with an error
        q.put((rank, "error: " + type(e).__name__))


def test_a_rank_that_leaves_ends_the_next_collective_with_an_error():
    """Failure detection without a GPU: rank 1 exits between steps; rank 0's
    next collective (the whole-job rate's max over ranks) raises within the
    process group's short timeout instead of hanging."""
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_leaves, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert procs[1].exitcode == 3
    assert procs[0].exitcode == 0
    rank, msg = q.get(timeout=5)
    assert rank == 0 and msg.startswith("error"), msg
