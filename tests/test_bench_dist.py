"""The N > 1 replica path of bench.py: whole-job units are summed and the time is
the maximum over ranks (gloo, world size 2, CPU only)."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, secs = bench.aggregate(units=1000.0 * (rank + 1), seconds=2.0 + rank, world=world)
    out[rank] = (units, secs)
    dist.destroy_process_group()


def test_aggregate_sums_units_and_takes_max_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (3000.0, 3.0)


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate(5.0, 2.0, 1) == (5.0, 2.0)


def test_dist_env_defaults(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
