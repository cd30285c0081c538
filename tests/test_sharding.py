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


# --------------------------------------------------------------------------
# One swarm split over ranks: the FP64 merge of its tally group sums.
# --------------------------------------------------------------------------
GROUPS = 32


def _synthetic_particles(n, id0, seed):
    """Per-particle results of a drifting swarm (id0 .. id0 + n - 1): times
    around 1 ns, drift along z with diffusion, counts and energy sums."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.5e-9, 1.5e-9, n)
    W = np.array([3e3, -1e3, 4e4])
    x = W[0] * t + rng.normal(0, 1e-6, n)
    y = W[1] * t + rng.normal(0, 1e-6, n)
    z = W[2] * t + rng.normal(0, 2e-6, n)
    n_real = np.full(n, 100, np.uint32)
    return {"x": x, "y": y, "z": z, "t": t, "sum_e": rng.uniform(200, 600, n), "sum_e2": rng.uniform(190, 590, n),
            "n_real": n_real, "n_null": rng.integers(0, 50, n).astype(np.uint32),
            "n_fail": np.zeros(n, np.uint32), "n_ion": rng.integers(0, 3, n).astype(np.uint32),
            "n_att": rng.integers(0, 2, n).astype(np.uint32), "steps": (n_real + rng.integers(50, 80, n)).astype(np.uint32),
            "status": np.zeros(n, np.uint32), "id": np.arange(id0, id0 + n, dtype=np.uint64)}


def _sums1(p):
    """Pass-1 group sums as bz.h lists them (count, x/t, y/t, z/t, G/z, D/z,
    x, y, z, t, energy sums, real, null, fail, G, D, incomplete, steps,
    stopped at t_end, removed), per batch group id mod 32."""
    import numpy as np
    x, y, z, t = p["x"], p["y"], p["z"], p["t"]
    G, D = p["n_ion"].astype(float), p["n_att"].astype(float)
    cols = [np.ones_like(t), x / t, y / t, z / t, G / z, D / z, x, y, z, t, p["sum_e"], p["sum_e2"],
            p["n_real"].astype(float), p["n_null"].astype(float), p["n_fail"].astype(float), G, D,
            np.zeros_like(t), p["steps"].astype(float), np.zeros_like(t), np.zeros_like(t)]
    g = (p["id"] % GROUPS).astype(int)
    out = np.zeros((GROUPS, 21))
    for q, c in enumerate(cols):
        np.add.at(out[:, q], g, c)
    return out


def _sums2(p, drift):
    """Pass-2 group sums about the drift vector (bz.h's list)."""
    import numpy as np
    x, y, z, t = p["x"], p["y"], p["z"], p["t"]
    dx, dy, dz = x - t * drift[0], y - t * drift[1], z - t * drift[2]
    dp2 = dx * dx + dy * dy
    d2 = dp2 + dz * dz
    fz, fx, fy = z - drift[5] * t, x - drift[3] * t, y - drift[4] * t
    cols = [d2 / t, dz * dz / (2 * t), dp2 / (4 * t), 2 * np.sqrt(d2), 2 * np.abs(dz), 2 * np.sqrt(dp2),
            fz * fz, fx * fx + fy * fy]
    g = (p["id"] % GROUPS).astype(int)
    out = np.zeros((GROUPS, 8))
    for q, c in enumerate(cols):
        np.add.at(out[:, q], g, c)
    return out


def _merge_worker(rank, world, port, n_total, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, b = sharding.id_range(rank, world, n_total)
    p = _synthetic_particles(b - a, a, seed=100 + rank)
    t = sharding.merge_tallies(_sums1(p), lambda d: _sums2(p, d), e_over_n_Td=50.0, n_total_m3=2.5e25,
                               nu_trial=1e13, error_flags=2 if rank == 1 else 0)
    out[rank] = t
    dist.destroy_process_group()


def test_one_swarm_over_two_gloo_ranks_merges_to_the_whole_swarm():
    """Two ranks hold two id ranges of one swarm; after the two all-reduces
    of the merge both hold the tallies of the whole swarm, equal to the
    oracle's estimators (Sec. 2.3) on all its electrons to FP64 rounding."""
    import numpy as np
    import torch.multiprocessing as mp
    from paper_1901_08140_gb300 import build as B
    from oracle import tallies as OT
    B.build()
    n_total = 5003
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_merge_worker, args=(2, port, n_total, out), nprocs=2, join=True, start_method="spawn")
    t0, t1 = out[0], out[1]
    assert t0 == t1
    parts = [_synthetic_particles(b - a, a, seed=100 + r)
             for r, (a, b) in enumerate(sharding.id_range(r, 2, n_total) for r in range(2))]
    whole = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    ref = OT.swarm_tallies(whole, 50.0, 2.5e25)
    for k in ("W", "Wx", "Wy", "W_flux", "eps", "eps_after", "alpha", "eta", "D", "D_L", "D_T", "sig", "sig_L",
              "sig_T", "D_L_flux", "D_T_flux", "mu", "efficiency", "lorentz_angle"):
        assert t0[k] == pytest.approx(ref[k], rel=1e-11, abs=1e-300), k
    for k in ("W_se", "eps_se", "D_L_se", "D_T_se", "sig_se"):
        assert t0[k] == pytest.approx(ref[k], rel=1e-8), k
    assert t0["n_particles"] == n_total and t0["n_real"] == 100 * n_total
    assert t0["error_flags"] == 2     # the parts' error bits are or-ed
    # one rank holding everything gives the same tallies
    from paper_1901_08140_gb300 import bz
    g1 = _sums1(whole)
    d = bz.drift_from_group_sums(g1)
    one = bz.finalize_group_sums(g1, _sums2(whole, d), 50.0, 2.5e25, 1e13)
    for k in ("W", "eps", "D_L", "D_T", "W_se", "D_T_se"):
        assert one[k] == pytest.approx(t0[k], rel=1e-12), k
