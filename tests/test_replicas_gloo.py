"""Multi-rank path of the benchmark on CPU (gloo, world size 2).

The hot path does not shard (every GPU runs an independent replica), so the
only cross-rank logic is the timing reduction: the job value is the sum of the
ranks' work divided by the slowest rank's time. This checks it with two gloo
ranks on 127.0.0.1, and that a rank that fails before the reduction makes the
other rank's collective end with an error instead of hanging (short timeout).
"""
import datetime
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _combine_worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=30))
    ms, units = bench.combine_ranks(dist, 10.0 + 5.0 * rank, 1000.0 * (rank + 1))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, units))


def test_combine_ranks_max_time_sum_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_combine_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, units in out:
        assert ms == 15.0 and units == 3000.0


def _failing_worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(3)  # the replica dies between steps, before the reduction
    try:
        bench.combine_ranks(dist, 1.0, 1.0)
        q.put("completed")
    except Exception as e:  # the collective ends with an error, it does not hang
        q.put("error: " + type(e).__name__)


def test_dead_rank_surfaces_as_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert procs[1].exitcode == 3
    msg = q.get(timeout=10)
    assert msg.startswith("error"), msg
