"""bench.py's multi-rank host logic on CPU (gloo, world size 2): every rank
takes rank 0's autotuned launch options, so the legs that follow take the
same branches (and meet at the same barriers) on every rank; a tuning done
on rank 0 alone broadcasts nothing."""
import argparse
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1901_08140_gb300 import autotune
    calls = []

    def fake_tune(ctx, mixes, cfgs, gas_lists=None):  # a tuning whose outcome differs per rank
        calls.append(rank)
        return {"window_c": 1.0 + rank, "tiles_per_block": 8 * (rank + 1), "blocks_per_sm": 0, "cached": False}

    autotune.tune = fake_tune
    args = argparse.Namespace(no_tune=False)
    shared = bench.tuned(None, None, None, args)
    alone = bench.tuned(None, None, None, args, shared=False)
    out[rank] = (shared, alone, list(calls))
    dist.destroy_process_group()


def test_ranks_share_rank0_tuning():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    (s0, a0, c0), (s1, a1, c1) = out[0], out[1]
    assert s0 == s1 == {"window_c": 1.0, "tiles_per_block": 8, "blocks_per_sm": 0, "cached": False}
    # the shared call tunes on rank 0 only; the unshared one tunes on each rank
    assert c0 == [0, 0] and c1 == [1]
    assert a1["window_c"] == 2.0 and a0["window_c"] == 1.0
