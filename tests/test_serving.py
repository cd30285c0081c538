"""Serving through the C ABI (bz_server_create, bz_submit, bz_poll,
bz_cancel): admission, grouping, ordering, cancellation and admission
overflow on a simulated server (host only, no device), and on the GPU each
request's result alone and in the mix."""
import time

import numpy as np
import pytest

from paper_1901_08140_gb300 import build as B
from paper_1901_08140_gb300 import bz
from paper_1901_08140_gb300 import serving as S

MIB = 1 << 20


@pytest.fixture(scope="module")
def L():
    B.build()
    return bz.lib()


def _cfg(n=1000, **kw):
    return bz.make_config(n_electrons=n, real_collisions=10, e_over_n_Td=10.0, **kw)


def _bytes(n):
    return 92 * n + 2 * MIB


def _wait_all(srv, ids, timeout=20.0):
    out, t0 = {}, time.time()
    while len(out) < len(ids):
        for rid in ids:
            if rid in out:
                continue
            r = srv.poll(rid)
            if r is not None:
                out[rid] = r
        assert time.time() - t0 < timeout, "the simulated server did not finish"
        time.sleep(1e-4)
    return out


def test_admission_respects_slots_budget_and_order(L):
    budget = _bytes(1000) * 2 + _bytes(500)  # two 1000-electron requests and a 500 one at once
    srv = S.Server(None, memory_budget=budget, n_slots=3, max_group=1, simulate=200)
    ids = [srv.submit(None, _cfg(n)) for n in (1000, 1000, 1000, 500, 2000)]
    res = _wait_all(srv, ids)
    st = srv.stats()
    assert st["completed"] == 5 and st["max_running"] <= 3
    assert st["peak_bytes_in_use"] <= budget
    # admission in submission order: launches are numbered in the order of the ids
    launches = [res[i][2]["launch"] for i in ids]
    assert launches == sorted(launches) and len(set(launches)) == 5
    # the third 1000-electron request had to wait for memory: admitted after another one ended
    assert res[ids[2]][2]["t_admit"] >= min(res[ids[0]][2]["t_done"], res[ids[1]][2]["t_done"])
    for rid, n in zip(ids, (1000, 1000, 1000, 500, 2000)):
        st_, t, info = res[rid]
        assert st_ == bz.BZ_OK and t["n_particles"] == n and t["n_real"] == 10 * n
        assert info["t_done"] >= info["t_admit"] >= info["t_submit"]
    srv.close()


def test_queued_requests_share_a_launch_within_budget(L):
    budget = _bytes(1000) * 3
    srv = S.Server(None, memory_budget=budget, n_slots=2, max_group=8, simulate=50)
    srv.pause()
    ids = [srv.submit(None, _cfg(1000)) for _ in range(7)]
    srv.pause(False)
    res = _wait_all(srv, ids)
    groups = {}
    for rid in ids:
        groups.setdefault(res[rid][2]["launch"], []).append(rid)
    sizes = [len(groups[k]) for k in sorted(groups)]
    assert sizes[0] == 3 and sum(sizes) == 7          # as many as the memory budget allows
    assert all(res[rid][2]["group_size"] == len(g) for g in groups.values() for rid in g)
    assert srv.stats()["peak_bytes_in_use"] <= budget
    srv.close()


def test_groups_hold_one_kernel_class_and_avalanches_run_alone(L):
    srv = S.Server(None, memory_budget=1e12, n_slots=1, max_group=8, simulate=20)
    cfgs = [_cfg(), _cfg(), _cfg(b_T=1.0), _cfg(b_T=0.5), _cfg(spawn=True, pop_cap=10 ** 4), _cfg(), _cfg(),
            _cfg(precision=64), _cfg(precision=64)]
    srv.pause()
    ids = [srv.submit(None, c) for c in cfgs]
    srv.pause(False)
    res = _wait_all(srv, ids)
    launch = [res[i][2]["launch"] for i in ids]
    # the head's class is gathered past other classes: [0, 1, 5, 6] lean without B,
    # [2, 3] with B, [4] spawn alone, [7, 8] FP64 -- each launch led by the oldest
    # request still queued
    assert launch == [0, 0, 1, 1, 2, 0, 0, 3, 3]
    srv.close()


def test_cancel_queued_running_and_finished_requests(L):
    srv = S.Server(None, memory_budget=1e12, n_slots=1, max_group=1, simulate=2000)
    a, b, c = (srv.submit(None, _cfg()) for _ in range(3))
    t0 = time.time()
    while srv.stats()["running"] == 0:     # a starts, b and c wait for the only slot
        assert time.time() - t0 < 5
        time.sleep(1e-4)
    srv.cancel(b)                           # queued: never starts
    srv.cancel(a)                           # running: its result is dropped
    assert srv.poll(a)[0] == bz.BZ_ECANCEL and srv.poll(b)[0] == bz.BZ_ECANCEL
    res = _wait_all(srv, [c])
    assert res[c][0] == bz.BZ_OK
    st = srv.stats()
    assert st["cancelled"] == 2 and st["completed"] == 1 and st["launches"] == 2
    assert st["bytes_in_use"] == 0 and st["running"] == 0
    d = srv.submit(None, _cfg())
    t0 = time.time()
    while srv.stats()["completed"] < 2:
        assert time.time() - t0 < 10
        time.sleep(1e-4)
    srv.cancel(d)                           # finished but not delivered: dropped
    assert srv.poll(d)[0] == bz.BZ_ECANCEL
    with pytest.raises(bz.BzError) as ei:   # delivered ids are forgotten
        srv.poll(d)
    assert ei.value.status == bz.BZ_EINVAL
    with pytest.raises(bz.BzError):
        srv.cancel(12345)
    srv.close()


def test_admission_overflow_is_rejected_at_submission(L):
    srv = S.Server(None, memory_budget=1e6, n_slots=2, simulate=5)
    with pytest.raises(bz.BzError) as ei:
        srv.submit(None, _cfg(10 ** 6))
    assert ei.value.status == bz.BZ_EBUDGET
    # spawn requests hold memory for their population cap
    with pytest.raises(bz.BzError) as ei:
        srv.submit(None, _cfg(1, spawn=True, pop_cap=10 ** 5))
    assert ei.value.status == bz.BZ_EBUDGET
    with pytest.raises(bz.BzError) as ei:     # invalid configurations never queue
        srv.submit(None, _cfg(0))
    assert ei.value.status == bz.BZ_EINVAL
    # ... among them bounded-wait settings out of range
    for bad in (dict(stage_wait_s=float("nan")), dict(stage_wait_s=4000.0), dict(hold_stage=2),
                dict(spawn_wait_s=float("inf")), dict(hold_pending=1)):
        with pytest.raises(bz.BzError) as ei:
            srv.submit(None, _cfg(10, **bad))
        assert ei.value.status == bz.BZ_EINVAL, bad
    assert srv.stats()["submitted"] == 0
    srv.close()


def test_server_options_out_of_range_are_rejected(L):
    for kw in (dict(max_group=70000), dict(n_slots=65), dict(simulate=-1)):
        opts = dict(memory_budget=1e9, n_slots=2, max_group=8, simulate=5)
        opts.update(kw)
        with pytest.raises(bz.BzError) as ei:
            S.Server(None, **opts)
        assert ei.value.status == bz.BZ_EINVAL, kw


def test_destroy_cancels_what_is_queued(L):
    srv = S.Server(None, memory_budget=1e12, n_slots=1, max_group=1, simulate=500)
    for _ in range(5):
        srv.submit(None, _cfg())
    srv.close()   # returns after the running launch ends; nothing leaks or hangs


def test_run_in_real_time_admits_arrivals_while_others_run(L):
    srv = S.Server(None, memory_budget=1e12, n_slots=4, max_group=1, simulate=3000)
    reqs = [S.Request(i, None, _cfg(), arrival=a, n_electrons=1000) for i, a in enumerate([0.0, 0.005, 0.01])]
    done = srv.run(reqs, realtime=True)
    by = {r.rid: r for r in done}
    assert by[1].admitted < by[0].done and by[2].admitted < by[0].done
    assert srv.stats()["max_running"] == 3
    srv.close()


def test_poisson_arrivals_and_summary():
    a = S.poisson_arrivals(1000.0, 20000, seed=3)
    gaps = np.diff(a)
    assert abs(gaps.mean() - 1e-3) < 3e-5 and np.all(gaps > 0)
    rs = [S.Request(i, None, None, arrival=x, n_electrons=1) for i, x in enumerate([0.0, 0.1, 0.2])]
    for r, d in zip(rs, [0.05, 0.2, 0.4]):
        r.done = d
        r.tallies = {"n_real": 10}
    s = S.latency_summary(rs)
    assert s["requests"] == 3 and abs(s["p50_ms"] - 100.0) < 1e-9


@pytest.mark.gpu
def test_results_are_the_same_alone_and_in_the_mix():
    """Through bz_submit / bz_poll: each request's tallies equal those of the
    swarm run alone (bz_run_swarm), bit for bit."""
    from paper_1901_08140_gb300 import workloads as W
    B.build()
    ctx = bz.Context(0)
    specs = W.batched_swarms(count=24, real_collisions=100, max_electrons=30000)
    mixes = [bz.Mixture(ctx, s.gases) for s in specs]
    cfgs = [bz.config_from_spec(s, trial_mode=bz.BZ_TRIAL_WINDOW if i % 2 else bz.BZ_TRIAL_LAZY)
            for i, s in enumerate(specs)]
    alone = []
    for m, c in zip(mixes, cfgs):
        sw = bz.run_swarm(ctx, m, c)
        alone.append(sw.tallies())
        sw.close()
    for slots, arrivals in ((8, [0.0] * len(cfgs)), (3, list(np.linspace(0.0, 0.02, len(cfgs))))):
        reqs = [S.Request(i, m, c, arrival=a, n_electrons=int(c.n_electrons))
                for i, (m, c, a) in enumerate(zip(mixes, cfgs, arrivals))]
        srv = S.Server(ctx, memory_budget=60e9, n_slots=slots, max_group=6)
        done = srv.run(reqs, realtime=True)
        assert srv.stats()["max_running"] > 1 and len(done) == len(reqs)
        for r in done:
            a = alone[r.rid]
            assert r.status == bz.BZ_OK
            for k in ("W", "eps", "D_L", "D_T", "n_real", "n_null", "n_window"):
                assert r.tallies[k] == a[k], (r.rid, k)
        srv.close()


@pytest.mark.gpu
def test_avalanche_requests_alone_and_in_the_mix():
    """Spawn-mode requests run in launches of their own beside batched swarms;
    the population they reach (integer counts, fixed by the ids' random
    numbers) is the same as when each runs alone."""
    from paper_1901_08140_gb300 import workloads as W
    B.build()
    ctx = bz.Context(0)
    specs = W.batched_swarms(count=8, real_collisions=100, max_electrons=20000)
    mixes = [bz.Mixture(ctx, s.gases) for s in specs]
    cfgs = [bz.config_from_spec(s, trial_mode=bz.BZ_TRIAL_WINDOW) for s in specs]
    ava = bz.Mixture(ctx, W.ar_co2_mixture())
    for i in range(3):
        mixes.insert(2 + 3 * i, ava)
        cfgs.insert(2 + 3 * i, bz.make_config(n_electrons=4, real_collisions=10 ** 9, e_over_n_Td=250.0,
                                              seed=W.swarm_seed(70 + i), t_end_s=0.2e-9, spawn=True,
                                              pop_cap=10 ** 6, trial_mode=bz.BZ_TRIAL_WINDOW))
    alone = []
    for m, c in zip(mixes, cfgs):
        sw = bz.run_swarm(ctx, m, c)
        alone.append(sw.tallies())
        sw.close()
    assert all(alone[2 + 3 * i]["n_spawned"] > 0 for i in range(3))
    reqs = [S.Request(i, m, c, arrival=a, n_electrons=int(c.n_electrons))
            for i, (m, c, a) in enumerate(zip(mixes, cfgs, np.linspace(0.0, 0.01, len(cfgs))))]
    srv = S.Server(ctx, memory_budget=60e9, n_slots=3, max_group=4)
    done = srv.run(reqs, realtime=True)
    assert len(done) == len(reqs)
    for r in done:
        a = alone[r.rid]
        for k in ("n_particles", "n_real", "n_ion", "n_att", "n_spawned", "n_alive", "n_capped"):
            assert r.tallies[k] == a[k], (r.rid, k)
        assert r.tallies["eps"] == pytest.approx(a["eps"], rel=1e-12, abs=0.0)
    srv.close()


@pytest.mark.gpu
def test_cancel_on_the_gpu_drops_only_the_cancelled_request():
    from paper_1901_08140_gb300 import workloads as W
    B.build()
    ctx = bz.Context(0)
    specs = W.batched_swarms(count=6, real_collisions=200, max_electrons=50000)
    mixes = [bz.Mixture(ctx, s.gases) for s in specs]
    cfgs = [bz.config_from_spec(s, trial_mode=bz.BZ_TRIAL_WINDOW) for s in specs]
    srv = S.Server(ctx, memory_budget=60e9, n_slots=1, max_group=2)
    srv.pause()
    ids = [srv.submit(m, c) for m, c in zip(mixes, cfgs)]
    srv.cancel(ids[1])
    srv.pause(False)
    while srv.stats()["running"] == 0:
        time.sleep(1e-4)
    srv.cancel(ids[0])
    res = _wait_all(srv, ids, timeout=120)
    for k, rid in enumerate(ids):
        if k in (0, 1):
            assert res[rid][0] == bz.BZ_ECANCEL
        else:
            sw = bz.run_swarm(ctx, mixes[k], cfgs[k])
            a = sw.tallies()
            sw.close()
            assert res[rid][0] == bz.BZ_OK and res[rid][1]["W"] == a["W"] and res[rid][1]["n_real"] == a["n_real"]
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()
