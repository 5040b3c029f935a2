"""world_size-2 gloo test of the multi-rank host logic (CPU): ranks get
distinct Philox keys and disjoint request slices, and the reported time is the
slowest rank's."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1310_3435_gb300 import replicas as R
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = R.rank_seed(7, rank)
        mine = R.shard(range(10), rank, world)
        t = 1.0 + rank                      # rank 1 is the slow one
        tmax = R.max_over_ranks(t)
        rate = R.whole_job_rate(100.0, world, tmax)
        q.put((rank, seed, mine, tmax, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_nothing_but_the_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, t0, v0), (r1, s1, m1, t1, v1) = out
    assert s0 != s1
    assert set(m0).isdisjoint(m1) and sorted(m0 + m1) == list(range(10))
    assert t0 == t1 == 2.0
    assert v0 == v1 == 100.0 * 2 / 2.0


def _dying_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import datetime
    import torch.distributed as dist
    from paper_1310_3435_gb300 import replicas as R
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)                         # the rank dies between steps
    try:
        R.max_over_ranks(1.0)
        q.put((rank, "no error"))
    except Exception as e:                  # the survivor learns of it, no hang
        q.put((rank, type(e).__name__))


def test_a_dead_rank_is_detected_by_the_timing_collective():
    """Failure detection on the host: rank 1 exits before the max-over-ranks
    collective; rank 0's collective ends with an error within the process
    group's timeout instead of waiting for ever."""
    import time
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    rank, what = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert rank == 0 and what != "no error", what
    assert procs[1].exitcode == 3
    assert time.time() - t0 < 100
