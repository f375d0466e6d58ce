"""bench.py's multi-rank path (replicas, no data-path collective): the job
time is the max over ranks and the value counts every rank's work.  Run as
two gloo ranks on the CPU."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    total = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (total, bench.throughput(world, 1000, 200, 5, total))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 150.0
    assert out[0][1] == 2 * 1000 * 200 * 5 / 0.150
