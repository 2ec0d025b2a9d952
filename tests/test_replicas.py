"""bench.py's multi-GPU path is replicas only: no collective on the data path,
one all-reduce (max) of the timed duration.  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
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


def _failing_worker(rank, world, port, q):
    # rank 1 fails between steps (before the timing exchange); rank 0 must get an
    # error from the collective within the process-group timeout, not hang
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        q.put((rank, "left"))
        q.close()
        q.join_thread()                           # the message is out before the process ends
        os._exit(3)
    import bench
    try:
        bench.aggregate_over_ranks(100.0, 5000)
        q.put((rank, "no error"))
    except Exception as exc:                      # gloo reports the lost peer
        q.put((rank, "error: " + type(exc).__name__))
    q.close()
    q.join_thread()
    os._exit(0)


def test_a_rank_that_leaves_is_detected_by_the_other():
    import time
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.perf_counter()
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert out[1] == "left"
    assert out[0].startswith("error"), out
    assert time.perf_counter() - t0 < 90
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0


def test_gpus_n_without_torchrun_starts_n_ranks_itself():
    """bench.py --gpus N (no torchrun) re-launches itself as N ranks through
    torch.distributed.run on 127.0.0.1, one per GPU; on a host with fewer GPUs
    it refuses cleanly (exit status 2, one line on stderr, no traceback)."""
    import subprocess
    import sys

    import bench
    cmd = bench.replica_command(["--gpus", "2", "--steps", "3"], 2, 29555)
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=2" in cmd and "--master-addr=127.0.0.1" in cmd and "--master-port=29555" in cmd
    assert cmd[-4:] == ["--gpus", "2", "--steps", "3"] and cmd[-5].endswith("bench.py")
    import torch
    if torch.cuda.is_available() and torch.cuda.device_count() >= 2:
        pytest.skip("this host has two GPUs: the refusal path does not apply")
    env = dict(os.environ)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, bench.__file__, "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 2, (r.returncode, r.stderr[-2000:])
    assert "needs 2 GPUs" in r.stderr and "Traceback" not in r.stderr
    assert r.stdout.strip() == ""


def test_parallelism_label_follows_the_world_size():
    import types

    import bench
    g = types.SimpleNamespace(n=10, m=20, s=0, t=9)
    wl = types.SimpleNamespace(describe=lambda: "tiny")
    args = types.SimpleNamespace(batch=5, gpus=4)
    assert bench.config_of(args, g, wl, 4)["parallelism"] == "replicas x4"
    assert bench.config_of(args, g, wl)["parallelism"] == "replicas x1"
