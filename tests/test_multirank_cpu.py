"""The N > 1 path of bench.py on CPU: two ranks over the gloo backend (one
replica per rank, no data-path collective).  The step time the job reports
is the maximum over ranks, the whole-job rate counts every rank's right-hand
sides, the reference arm runs on rank 0 only, and a rank that dies before the
timing collective makes the surviving rank's collective fail instead of hang."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.dist_max(100.0 + 7.0 * rank)
    dist.barrier()
    q.put((rank, ms, bench.whole_job_rate(world, 32, ms)))
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_step():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [107.0, 107.0]
    assert all(o[2] == pytest.approx(2 * 32 / 0.107) for o in out)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_max(3.5) == 3.5
    assert bench.whole_job_rate(1, 32, 500.0) == pytest.approx(64.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def _rank_dies(rank, world, port, q):
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=15))
    import bench
    if rank == 1:
        os._exit(3)  # this replica fails between steps, before the timing all-reduce
    try:
        bench.dist_max(1.0)
        q.put("completed")
    except Exception as e:  # the collective reports the lost peer
        q.put("error " + type(e).__name__)


def test_surviving_rank_sees_a_failed_peer():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_dies, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    msg = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert msg.startswith("error"), msg
    assert procs[1].exitcode == 3

