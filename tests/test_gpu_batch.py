"""Batched swarms (one persistent launch over many swarms, CUDA graph):
every swarm's results equal those of its own bz_run_swarm."""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1901_08140_gb300 import bz
from paper_1901_08140_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1901_08140_gb300 import build as B
    B.build()
    c = bz.Context(0)
    yield c
    c.close()


def _items(ctx):
    gases = {"ar": [W.argon_like()], "arco2": W.ar_co2_mixture(), "r1": W.batched_swarms(count=3)[1].gases,
             "r2": W.batched_swarms(count=3)[2].gases}
    mixes = {k: bz.Mixture(ctx, g) for k, g in gases.items()}
    spec = [("ar", 1, 10.0, 0.0, 0.0, 0), ("arco2", 33, 100.0, 1.0, math.pi / 2, 0), ("r1", 1000, 50.0, 0.5, 1.0, 2),
            ("ar", 5000, 300.0, 0.0, 0.0, 2), ("r2", 20000, 5.0, 1.5, 2.5, 2), ("arco2", 4097, 20.0, 0.0, 0.0, 0),
            ("r1", 257, 700.0, 0.0, 0.0, 2), ("ar", 3000, 1.0, 2.0, 0.3, 2)]
    items = []
    for i, (mk, n, eon, b, ang, mode) in enumerate(spec):
        cfg = bz.make_config(n_electrons=n, real_collisions=60, e_over_n_Td=eon, b_T=b, b_angle_rad=ang,
                             seed=W.swarm_seed(900 + i), trial_mode=mode, id_offset=7 * i)
        items.append((mixes[mk], cfg))
    return items


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("field", [True, False])
@pytest.mark.parametrize("staged", [True, False])
def test_batch_equals_individual_runs(ctx, use_graph, field, staged):
    """A batch runs one build of the step kernel; batches whose swarms all
    have (or all lack) a magnetic field, and whose mixtures all stage (or all
    leave in global memory) their channel tables, run the build each swarm
    runs alone, so every value is the same bit for bit."""
    items = [(m, c) for m, c in _items(ctx)
             if (c.b_T > 0) == field and bool(m.info["channels_in_smem"]) == staged]
    assert items
    batch = bz.Batch(ctx, [m for m, _ in items], [c for _, c in items], tile_particles=512, use_graph=use_graph)
    batch.launch()
    bt = batch.tallies()
    for i, (mix, cfg) in enumerate(items):
        sw = bz.run_swarm(ctx, mix, cfg)
        t = sw.tallies()
        p = sw.particles()
        sw.close()
        q = batch.particles(i)
        for k in ["x", "y", "z", "t", "sum_e", "sum_e2", "n_real", "n_null", "n_fail", "n_ion", "n_att", "steps"]:
            assert np.array_equal(p[k], q[k]), (i, k)
        for k in ["W", "eps", "D_L", "D_T", "W_se", "alpha", "efficiency"]:
            assert bt[i][k] == t[k] or (math.isnan(t[k]) and math.isnan(bt[i][k])), (i, k)
        assert bt[i]["n_real"] == t["n_real"] and bt[i]["error_flags"] == 0
    km, tm = batch.timing()
    assert km > 0 and tm > 0
    batch.close()


@pytest.mark.parametrize("block", [128, 384, 768])
@pytest.mark.parametrize("field", [True, False])
@pytest.mark.parametrize("staged", [True, False])
def test_block_sizes_give_the_same_results(ctx, block, field, staged):
    """Blocks of 128, 384 or 768 threads run the same step kernel at the same
    register cap: electrons are independent and every draw is keyed by the
    electron's id, so every value equals the 256-thread launch's bit for bit,
    batched and alone."""
    items = [(m, c) for m, c in _items(ctx)
             if (c.b_T > 0) == field and bool(m.info["channels_in_smem"]) == staged]
    ref = bz.Batch(ctx, [m for m, _ in items], [c for _, c in items], tile_particles=512)
    ref.launch()
    rt = ref.tallies()
    got = bz.Batch(ctx, [m for m, _ in items], [c for _, c in items], tile_particles=512, block_threads=block)
    got.launch()
    gt = got.tallies()
    for i, (mix, cfg) in enumerate(items):
        p, q = ref.particles(i), got.particles(i)
        for k in ["x", "y", "z", "t", "sum_e", "sum_e2", "n_real", "n_null", "n_fail", "n_ion", "n_att", "steps"]:
            assert np.array_equal(p[k], q[k]), (i, k)
        for k in ["W", "eps", "D_L", "D_T", "W_se", "alpha", "efficiency"]:
            assert gt[i][k] == rt[i][k] or (math.isnan(rt[i][k]) and math.isnan(gt[i][k])), (i, k)
        assert gt[i]["error_flags"] == 0
    mix, cfg = items[-1]
    alone = bz.run_swarm(ctx, mix, _with(cfg, block_threads=block))
    pa = alone.particles()
    alone.close()
    q = got.particles(len(items) - 1)
    for k in ["x", "t", "sum_e", "n_real", "n_null", "steps"]:
        assert np.array_equal(pa[k], q[k]), k
    ref.close()
    got.close()


def _with(cfg, **over):
    """A copy of a swarm configuration with some fields replaced."""
    out = bz.bz_swarm_config()
    C.memmove(C.byref(out), C.byref(cfg), C.sizeof(bz.bz_swarm_config))
    for k, v in over.items():
        setattr(out, k, v)
    return out


def test_table_budget_gives_the_same_results(ctx):
    """Mixtures compiled for one block per SM (a larger table budget: a
    denser bucket index, every bin maximum in shared memory) locate the same
    records and bin maxima, so a batch of 768-thread blocks on them gives the
    default batch's values bit for bit (both leave the channel tables in
    global memory)."""
    import dataclasses
    from paper_1901_08140_gb300 import autotune
    specs = [dataclasses.replace(s, n_electrons=min(s.n_electrons, 2000))
             for s in W.batched_swarms(count=64, real_collisions=50)]
    small = [bz.Mixture(ctx, s.gases) for s in specs]
    big = autotune.mixtures_for(ctx, [s.gases for s in specs], {"smem_budget": autotune.ONE_BLOCK_BUDGET})
    keep = [i for i in range(len(specs)) if small[i].info["channels_in_smem"] == big[i].info["channels_in_smem"] == 0]
    assert keep
    assert any(big[i].info["smem_bytes"] > small[i].info["smem_bytes"] for i in keep)  # some layouts differ
    cfgs = [bz.config_from_spec(specs[i], trial_mode=bz.BZ_TRIAL_WINDOW) for i in keep]
    ref = bz.Batch(ctx, [small[i] for i in keep], cfgs)
    got = bz.Batch(ctx, [big[i] for i in keep], cfgs, block_threads=768)
    ref.launch()
    got.launch()
    rt, gt = ref.tallies(), got.tallies()
    for j in range(len(keep)):
        p, q = ref.particles(j), got.particles(j)
        for k in ["x", "y", "z", "t", "sum_e", "sum_e2", "n_real", "n_null", "n_fail", "steps"]:
            assert np.array_equal(p[k], q[k]), (j, k)
        for k in ["W", "eps", "D_L", "D_T", "W_se"]:
            assert gt[j][k] == rt[j][k], (j, k)
    ref.close()
    got.close()
    for m in small + big:
        m.close()


def test_unsupported_block_sizes_are_rejected(ctx):
    mix, cfg = _items(ctx)[3]
    for bad in (64, 192, 512, 1024):
        with pytest.raises(bz.BzError, match="block_threads"):
            bz.Batch(ctx, [mix], [cfg], block_threads=bad)
        with pytest.raises(bz.BzError, match="block_threads"):
            bz.run_swarm(ctx, mix, _with(cfg, block_threads=bad))
    c64 = _with(cfg, precision=64)
    with pytest.raises(bz.BzError, match="128, 384 or 768"):
        bz.Batch(ctx, [mix], [c64], block_threads=128)
    with pytest.raises(bz.BzError, match="128, 384 or 768"):
        bz.run_swarm(ctx, mix, _with(c64, block_threads=384))
    cv = _with(cfg, trial_mode=bz.BZ_TRIAL_VARIABLE)
    with pytest.raises(bz.BzError, match="128, 384 or 768"):
        bz.Batch(ctx, [mix], [cv], block_threads=128)


def test_mixed_field_batch(ctx):
    """Swarms without a field batched with swarms with one run the field's
    build: the field swarms match their runs alone bit for bit, the others
    to FP32 rounding along their trajectories (statistics within errors)."""
    items = _items(ctx)
    batch = bz.Batch(ctx, [m for m, _ in items], [c for _, c in items], tile_particles=512)
    batch.launch()
    bt = batch.tallies()
    for i, (mix, cfg) in enumerate(items):
        sw = bz.run_swarm(ctx, mix, cfg)
        t = sw.tallies()
        sw.close()
        assert bt[i]["n_real"] == t["n_real"]
        if cfg.b_T > 0:
            assert bt[i]["W"] == t["W"] and bt[i]["n_null"] == t["n_null"], i
        elif cfg.n_electrons > 100:
            for k in ("W", "eps"):
                assert abs(bt[i][k] - t[k]) <= 3 * math.hypot(bt[i][k + "_se"], t[k + "_se"]), (i, k)
    batch.close()


def test_mixed_staging_batch(ctx):
    """Mixtures that stage their channel tables batched with mixtures that
    cannot: the batch searches every mixture's cumulative table in global
    memory, so the staging mixtures' swarms match their runs alone in counts
    and statistically (a channel choice may differ where a draw falls within
    FP32 rounding of a boundary); the others bit for bit."""
    items = [(m, c) for m, c in _items(ctx) if c.b_T == 0]
    assert len({bool(m.info["channels_in_smem"]) for m, _ in items}) == 2
    batch = bz.Batch(ctx, [m for m, _ in items], [c for _, c in items], tile_particles=512)
    batch.launch()
    bt = batch.tallies()
    for i, (mix, cfg) in enumerate(items):
        sw = bz.run_swarm(ctx, mix, cfg)
        t = sw.tallies()
        sw.close()
        assert bt[i]["n_real"] == t["n_real"] and bt[i]["n_particles"] == t["n_particles"]
        if not mix.info["channels_in_smem"]:
            assert bt[i]["W"] == t["W"] and bt[i]["n_null"] == t["n_null"], i
        elif cfg.n_electrons > 100:
            for k in ("W", "eps"):
                assert abs(bt[i][k] - t[k]) <= 3 * math.hypot(bt[i][k + "_se"], t[k + "_se"]), (i, k)
    batch.close()


def test_channel_tables_in_l2_policy(ctx):
    """The staging policy that keeps every channel table in global memory
    (the cumulative-table search) runs the same swarms: equal counts,
    swarm statistics within their errors, and equal to a batch whose
    mixtures cannot stage their channels bit for bit."""
    items = [(m, c) for m, c in _items(ctx) if c.b_T == 0]
    staged = [(m, c) for m, c in items if m.info["channels_in_smem"]]
    a = bz.Batch(ctx, [m for m, _ in staged], [c for _, c in staged], tile_particles=512)
    b = bz.Batch(ctx, [m for m, _ in staged], [c for _, c in staged], tile_particles=512, channels_in_l2=True)
    a.launch()
    b.launch()
    ta, tb = a.tallies(), b.tallies()
    for i, (_, cfg) in enumerate(staged):
        assert ta[i]["n_real"] == tb[i]["n_real"] and ta[i]["n_particles"] == tb[i]["n_particles"]
        if cfg.n_electrons > 100:
            for k in ("W", "eps"):
                assert abs(ta[i][k] - tb[i][k]) <= 3 * math.hypot(ta[i][k + "_se"], tb[i][k + "_se"]), (i, k)
    a.close()
    b.close()
    # a mixed batch already searches in global memory: the policy changes nothing there
    c = bz.Batch(ctx, [m for m, _ in items], [c for _, c in items], tile_particles=512)
    d = bz.Batch(ctx, [m for m, _ in items], [c for _, c in items], tile_particles=512, channels_in_l2=True)
    c.launch()
    d.launch()
    assert [t["W"] for t in c.tallies()] == [t["W"] for t in d.tallies()]
    c.close()
    d.close()


def test_batch_relaunch_is_reproducible(ctx):
    items = _items(ctx)
    batch = bz.Batch(ctx, [m for m, _ in items], [c for _, c in items])
    batch.launch()
    a = batch.tallies()
    pa = batch.particles(4)
    batch.launch()
    b = batch.tallies()
    pb = batch.particles(4)
    assert all(x["W"] == y["W"] and x["n_null"] == y["n_null"] for x, y in zip(a, b))
    assert np.array_equal(pa["z"], pb["z"])
    batch.close()


def test_batch_rejects_mixed_precision(ctx):
    items = _items(ctx)[:2]
    cfgs = [c for _, c in items]
    cfgs[1].precision = 64
    with pytest.raises(bz.BzError) as ei:
        bz.Batch(ctx, [m for m, _ in items], cfgs)
    assert ei.value.status == bz.BZ_EINVAL
    # one tally grid row per swarm: at most 65535 swarms
    m, c = items[0]
    with pytest.raises(bz.BzError) as ei:
        bz.Batch(ctx, [m] * 65536, [c] * 65536)
    assert ei.value.status == bz.BZ_EINVAL


def test_set_up_does_not_wait_for_a_running_launch(ctx):
    """The library's set-up copies (a mixture's tables, a batch's descriptors)
    run on a stream of their own: while a launch runs on the legacy default
    stream, compiling and uploading a mixture and setting up a batch return
    before it ends (the overlap the end-to-end loop relies on)."""
    import time
    specs = W.argon_sweep(n_electrons=1_000_000, real_collisions=1000, points=32)
    mix = bz.Mixture(ctx, specs[0].gases)
    cfgs = [bz.config_from_spec(s, trial_mode=bz.BZ_TRIAL_WINDOW) for s in specs]
    other = W.batched_swarms(count=2)[1]
    ocfg = bz.config_from_spec(other, n_electrons=1000, real_collisions=10, trial_mode=bz.BZ_TRIAL_WINDOW)
    # warm the allocators' caches with the same sizes first: a fresh pinned or
    # device allocation may itself wait for the device
    for _ in range(2):
        m = bz.Mixture(ctx, other.gases)
        b = bz.Batch(ctx, [m], [ocfg])
        b.close()
        m.close()
    big = bz.Batch(ctx, [mix] * len(cfgs), cfgs)
    big.launch()
    t0 = time.perf_counter()
    m2 = bz.Mixture(ctx, other.gases)
    b2 = bz.Batch(ctx, [m2], [ocfg])
    dt = time.perf_counter() - t0
    running = not big.ready()
    big.tallies()
    ms = big.timing()[0]
    b2.launch()
    t2 = b2.tallies()[0]
    assert running, f"the {ms:.0f} ms launch ended before the set-up returned ({dt * 1e3:.0f} ms)"
    assert dt < 0.5 * ms / 1e3
    assert t2["n_real"] == 10 * 1000
    b2.close()
    m2.close()
    big.close()
