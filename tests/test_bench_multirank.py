"""The multi-replica aggregation of bench.py on a world-size-2 gloo group
(CPU): the job time is the slowest rank's, the node count the sum."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    ms = [10.0, 12.5][rank]
    e2e = [0.2, 0.1][rank]
    res = bench.aggregate(ms, 1000 + rank, 5, e2e, dist, "cpu")
    out.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ms_max, total, value, e2e = res[r]
        assert ms_max == 12.5 and total == 2001.0
        assert value == pytest.approx(2001 * 5 / 12.5e-3 / 1e6)
        assert e2e == pytest.approx(2001 / 0.2 / 1e6)
