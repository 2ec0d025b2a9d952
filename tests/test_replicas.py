"""bench.py's multi-GPU path is replicas only: no collective on the data path,
one all-reduce (max) of the timed duration.  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, tot_ms, ws = bench.aggregate_over_ranks(100.0 * (rank + 1), 5000)
    q.put((rank, value, tot_ms, ws))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tot_ms, ws in out:
        assert ws == 2
        assert tot_ms == 200.0                      # the slower rank's time
        assert value == pytest.approx(2 * 5000 / 0.2)


def test_single_process_aggregate():
    import bench
    value, tot_ms, ws = bench.aggregate_over_ranks(50.0, 1000)
    assert ws == 1 and tot_ms == 50.0 and value == pytest.approx(20000.0)
