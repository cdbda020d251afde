"""Host logic of bench.py's N > 1 path (replicas), on CPU with gloo ranks.

Each rank runs an independent replica of the single-GPU solver; the whole-job
value is the units of all ranks over the slowest rank's time.  Here two gloo
ranks feed known units and times through the same aggregation code."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), HS3D_DIST_BACKEND="gloo")
    import bench
    w, r, _ = bench.dist_init()
    assert (w, r) == (world, rank)
    units = 1000.0 * (rank + 1)           # ranks process different amounts
    secs = 2.0 + rank                     # and take different times
    bench.barrier(w)
    val, slowest = bench.aggregate(units, secs, w)
    q.put((rank, val, slowest))
    dist.destroy_process_group()


def test_two_rank_aggregation_is_sum_over_max():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for _, val, slowest in res:
        assert slowest == 3.0
        assert abs(val - 3000.0 / 3.0) < 1e-9
