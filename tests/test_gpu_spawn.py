"""Spawn mode on the GPU: ionizations create electrons, attachments remove
them (Sec. 2), checked against closed forms and against the oracle."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1901_08140_gb300 import bz
from paper_1901_08140_gb300 import workloads as W
from test_oracle_pins import _const_rate_gas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1901_08140_gb300 import build as B
    B.build()
    c = bz.Context(0)
    yield c
    c.close()


def _run(ctx, gases, **kw):
    mix = bz.Mixture(ctx, gases)
    sw = bz.run_swarm(ctx, mix, bz.make_config(**kw))
    t = sw.tallies()
    p = sw.particles()
    sw.close()
    return t, p


@pytest.mark.parametrize("mode", [bz.BZ_TRIAL_LAZY, bz.BZ_TRIAL_WINDOW])
def test_yule_growth_on_gpu(ctx, mode):
    nu_i = 1e11
    n0, t_end = 20000, 3.0 / nu_i
    t, p = _run(ctx, [_const_rate_gas(1e12, nu_ion=nu_i)], n_electrons=n0, real_collisions=10 ** 9,
                e_over_n_Td=50.0, seed=21, t_end_s=t_end, spawn=True, pop_cap=2_000_000, trial_mode=mode)
    total = len(p["t"])
    expect = n0 * math.exp(nu_i * t_end)
    sd = math.sqrt(n0 * math.exp(nu_i * t_end) * (math.exp(nu_i * t_end) - 1))
    assert abs(total - expect) < 4 * sd
    assert t["n_spawned"] == total - n0 == int(p["n_ion"].sum())
    assert t["n_alive"] == total and t["n_capped"] == 0 and t["error_flags"] == 0
    assert np.allclose(p["t_birth"] + p["t"], t_end, rtol=1e-6, atol=0)
    assert len(np.unique(p["id"])) == total


def test_attachment_removes_on_gpu(ctx):
    nu_a = 1e11
    n0, t_end = 100000, 1.5 / nu_a
    t, p = _run(ctx, [_const_rate_gas(1e12, nu_att=nu_a)], n_electrons=n0, real_collisions=10 ** 9,
                e_over_n_Td=10.0, seed=5, t_end_s=t_end, spawn=True, pop_cap=n0)
    q = math.exp(-nu_a * t_end)
    assert abs(t["n_alive"] - n0 * q) < 4 * math.sqrt(n0 * q * (1 - q))
    assert t["n_removed"] == n0 - t["n_alive"] == int(np.sum(p["status"] == bz.ST_ATTACHED))


def test_spawn_fp64_matches_oracle_electron_by_electron(ctx):
    gases = W.ar_co2_mixture()
    kw = dict(e_over_n_Td=400.0, real_collisions=10 ** 6, seed=77, t_end_s=3e-11)
    n0, cap = 300, 100000
    t, p = _run(ctx, gases, n_electrons=n0, precision=64, spawn=True, pop_cap=cap, **kw)
    m = O.Mixture(gases)
    po = O.run_swarm_spawn(m, n=n0, pop_cap=cap, t_end=kw["t_end_s"], e_over_n_Td=kw["e_over_n_Td"],
                           real_collisions=kw["real_collisions"], seed=kw["seed"])
    assert len(po["id"]) > 2 * n0   # the avalanche grew
    og = {int(i): k for k, i in enumerate(p["id"])}
    oo = {int(i): k for k, i in enumerate(po["id"])}
    common = set(og) & set(oo)
    assert len(common) >= 0.95 * max(len(og), len(oo))
    same = 0
    for i in common:
        a, b = og[i], oo[i]
        if all(p[k][a] == po[k][b] for k in ("n_real", "n_null", "n_ion", "n_att", "steps", "status")):
            same += 1
            assert abs(p["t_birth"][a] - po["t_birth"][b]) <= 1e-9 * kw["t_end_s"]
            assert abs(p["z"][a] - po["z"][b]) <= 1e-9 * (abs(po["z"][b]) + 1e-12)
    assert same >= 0.95 * len(common)


def test_population_cap(ctx):
    nu_i = 1e11
    t, p = _run(ctx, [_const_rate_gas(1e12, nu_ion=nu_i)], n_electrons=1000, real_collisions=10 ** 9,
                e_over_n_Td=50.0, seed=3, t_end_s=5.0 / nu_i, spawn=True, pop_cap=20000)
    assert len(p["t"]) == 20000 and t["n_capped"] > 0
    assert int(p["n_ion"].sum()) == t["n_spawned"] + t["n_capped"]


def test_population_cap_at_the_start(ctx):
    """pop_cap equal to the primaries: every ionization is capped, none is created."""
    nu_i = 1e11
    t, p = _run(ctx, [_const_rate_gas(1e12, nu_ion=nu_i)], n_electrons=5000, real_collisions=10 ** 9,
                e_over_n_Td=50.0, seed=4, t_end_s=2.0 / nu_i, spawn=True, pop_cap=5000)
    assert len(p["t"]) == 5000 and t["n_spawned"] == 0
    assert t["n_capped"] == int(p["n_ion"].sum()) > 0


def test_spawn_is_reproducible_run_to_run(ctx):
    """Lanes take created electrons in whatever order they are published, yet
    each electron's history depends only on its id: two runs agree."""
    kw = dict(n_electrons=4, real_collisions=10 ** 9, e_over_n_Td=300.0, seed=31, t_end_s=0.25e-9, spawn=True,
              pop_cap=10 ** 6, trial_mode=bz.BZ_TRIAL_WINDOW)
    t1, p1 = _run(ctx, W.ar_co2_avalanche_mixture(), **kw)
    t2, p2 = _run(ctx, W.ar_co2_avalanche_mixture(), **kw)
    assert len(p1["id"]) > 100 and t1["n_capped"] == 0
    o1, o2 = np.argsort(p1["id"]), np.argsort(p2["id"])
    assert np.array_equal(p1["id"][o1], p2["id"][o2])
    for k in ("n_real", "n_null", "n_ion", "n_att", "steps", "status", "x", "z", "t", "t_birth"):
        assert np.array_equal(p1[k][o1], p2[k][o2]), k
    for k in ("n_particles", "n_real", "n_ion", "n_spawned", "n_alive"):
        assert t1[k] == t2[k]
    assert t1["W"] == pytest.approx(t2["W"], rel=1e-12, abs=0.0)


def test_avalanche_request_shape(ctx):
    """A 1 ns avalanche in the Ar/CO2-like mixture at 300 Td from one seed of electrons."""
    t, p = _run(ctx, W.ar_co2_mixture(), n_electrons=100, real_collisions=10 ** 9, e_over_n_Td=300.0, seed=9,
                t_end_s=1e-9, spawn=True, pop_cap=5_000_000, trial_mode=bz.BZ_TRIAL_WINDOW)
    assert t["n_particles"] == len(p["t"]) > 100
    assert t["n_alive"] + t["n_removed"] + t["n_incomplete"] == len(p["t"])
    assert t["error_flags"] == 0 and math.isfinite(t["W"]) and t["W"] > 0


def test_batch_rejects_spawn(ctx):
    mix = bz.Mixture(ctx, [W.argon_like()])
    cfg = bz.make_config(n_electrons=10, real_collisions=10, e_over_n_Td=10.0, spawn=True)
    with pytest.raises(bz.BzError):
        bz.Batch(ctx, [mix], [cfg])


def test_spawn_wait_gives_up_after_its_limit(ctx):
    """A failure made on the host: one electron is counted as pending but is
    never created, so lanes that run out of work keep waiting for it.  After
    spawn_wait_s the kernel gives up, flags BZ_ERR_SPAWN_WAIT, and returns:
    bz_read_tallies reports BZ_ETIMEOUT, every electron that existed was run
    (the counts equal the same swarm's run without the reservation), and the
    context stays usable."""
    import time
    mix = bz.Mixture(ctx, W.ar_co2_avalanche_mixture())
    kw = dict(n_electrons=64, real_collisions=10 ** 9, e_over_n_Td=300.0, seed=W.swarm_seed(91), t_end_s=0.05e-9,
              spawn=True, pop_cap=10 ** 4, trial_mode=bz.BZ_TRIAL_WINDOW)
    ref = bz.run_swarm(ctx, mix, bz.make_config(**kw))
    tr = ref.tallies()
    ref.close()
    t0 = time.time()
    sw = bz.run_swarm(ctx, mix, bz.make_config(spawn_wait_s=0.2, hold_pending=1, **kw))
    with pytest.raises(bz.BzError) as ei:
        sw.tallies()
    elapsed = time.time() - t0
    assert ei.value.status == bz.BZ_ETIMEOUT
    t = sw.tallies(check=False)
    sw.close()
    assert t["error_flags"] & bz.BZ_ERR_SPAWN_WAIT
    assert 0.2 <= elapsed < 30.0
    for k in ("n_particles", "n_real", "n_ion", "n_spawned", "n_alive"):
        assert t[k] == tr[k], k
    # the context still runs work
    ok = bz.run_swarm(ctx, mix, bz.make_config(n_electrons=1000, real_collisions=20, e_over_n_Td=50.0))
    assert ok.tallies()["n_real"] == 20000
    ok.close()
