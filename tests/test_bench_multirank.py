"""The multi-GPU bench path on the host: each rank times its own problem, the
job time is the slowest rank's (all-reduce MAX), and the whole-job value counts
the work of every rank.  Two gloo ranks on CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.0 + rank, 2.0 + 3 * rank]           # rank 1 is the slower one
        t, e = bench.max_over_ranks(mine, world, "cpu")
        q.put((rank, t, e, bench.whole_job_rate(100.0, world, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, e, rate in out:
        assert t == 2.0 and e == 5.0                   # max over ranks on every rank
        assert rate == pytest.approx(2 * 100.0 / 2.0)  # both ranks' work over the job time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
