"""The bench's multi-rank host logic on CPU ranks (gloo, world size 2): the
reductions behind the whole-job value (max of the ranks' times, sum of their
work) and the detection of a rank that leaves without reaching the barrier,
through a short process-group timeout.  No GPU is involved."""
import datetime
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = torch.multiprocessing


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reductions(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=30))
    mx = bench.max_over_ranks(dist, 1.5 + rank)
    sm = bench.sum_over_ranks(dist, 1.5 + rank)
    bench.barrier(dist)
    q.put((rank, mx, sm))
    dist.destroy_process_group()


def _one_rank_leaves(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=3))
    if rank == 1:
        q.put((rank, "left"))
        q.close()
        q.join_thread()                  # flush the message, then leave between
        os._exit(0)                      # steps with nothing in flight
    try:
        bench.barrier(dist)
        q.put((rank, "no error"))
    except Exception as e:               # the lost peer surfaces as an error, not a hang
        q.put((rank, "error: " + type(e).__name__))


def _run(target, world=2, timeout=90):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=timeout) for _ in range(world)]
    for p in ps:
        p.join(timeout=timeout)
        if p.is_alive():
            p.kill()
    return dict((o[0], o[1:]) for o in out)


def test_whole_job_reductions_over_two_cpu_ranks():
    res = _run(_reductions)
    for r in range(2):
        assert res[r] == (2.5, 4.0), res


def test_a_rank_that_leaves_is_detected_by_the_timeout():
    res = _run(_one_rank_leaves)
    assert res[1] == ("left",)
    assert res[0][0].startswith("error"), res
