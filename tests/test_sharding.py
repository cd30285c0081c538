"""Multi-rank host logic of the sharded path, on CPU with gloo (world size 2)."""
import os
import socket

import pytest

from paper_1901_08140_gb300 import sharding


def test_id_ranges_cover_exactly_once():
    for n, w in [(10, 2), (11, 2), (7, 3), (1, 4), (1000003, 8)]:
        ranges = [sharding.id_range(r, w, n) for r in range(w)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        assert all(ranges[i][1] == ranges[i + 1][0] for i in range(w - 1))
        sizes = [b - a for a, b in ranges]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.id_range(2, 2, 10)
    assert sharding.weak_offset(3, 1000) == 3000


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = sharding.reduce_step(10.0 + 5.0 * rank, 100.0 * (rank + 1))
    out[rank] = (ms, units)
    dist.destroy_process_group()


def test_max_time_and_summed_units_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1] == (15.0, 300.0)


def test_single_process_passthrough():
    assert sharding.reduce_step(3.0, 7.0) == (3.0, 7.0)
