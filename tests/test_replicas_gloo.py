"""The multi-GPU form is replicas only (independent problems per rank, no
collective on the data path): bench.py's timing aggregation takes the slowest
rank's time and counts every rank's points.  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]          # rank 1 is the slow one
    nodes = [1000, 1000][rank]
    got = bench.aggregate_timing(ms, nodes, 4, world, tdist, "cpu")
    out.put((rank, got))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_all_points():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ms, value = res[r]
        assert ms == 20.0
        assert value == pytest.approx(2 * 1000 * 4 / 20.0e-3)


def test_single_rank_is_unchanged():
    import bench
    assert bench.aggregate_timing(10.0, 500, 2, 1) == (10.0, 500 * 2 / 10.0e-3)
