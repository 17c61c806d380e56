"""The bench's multi-rank aggregation (one independent instance per rank, no
collective on the data path) with world size 2 over gloo on the CPU: the job's
step time is the slowest rank's and its work the sum of every rank's."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_ms = [120.0, 180.0][rank]
    samples = [1e9, 2e9][rank]
    backups = [5e8, 7e8][rank]
    res = bench.aggregate(t_ms, samples, backups, world, "cpu")
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_over_gloo():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        t, smp, bk = res[rank]
        assert t == 180.0
        assert smp == 3e9 and bk == 1.2e9
    # whole-job throughput = all ranks' samples / the slowest rank's time
    t, smp, _ = res[0]
    assert smp / (t / 1e3) == pytest.approx(3e9 / 0.18)


def test_single_rank_aggregation_is_identity():
    import bench
    assert bench.aggregate(10.0, 5.0, 2.0, 1, "cpu") == (10.0, 5.0, 2.0)
