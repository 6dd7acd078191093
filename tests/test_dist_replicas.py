"""The N-GPU bench runs independent replicas (the projection does not shard):
each rank projects its own batch and the job time is the slowest rank's.
Host logic checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_env()
    seconds = (0.5, 0.8)[rank]  # this rank's own timed region
    t = bench.slowest_rank(seconds, dist, device="cpu")
    q.put((r, w, local, t, bench.job_throughput(1000, 10, w, t)))
    dist.destroy_process_group()


def test_replicas_report_the_slowest_rank():
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
    assert [o[0] for o in out] == [0, 1]
    for r, w, local, t, v in out:
        assert w == 2 and local == r
        assert t == 0.8                      # the slowest rank's time, on every rank
        assert v == 1000 * 10 * 2 / 0.8      # all ranks' points over that time


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank(1.25, None) == 1.25
    assert bench.job_throughput(16, 3, 1, 2.0) == 24.0
