"""Serving loop: host-side admission and ordering with a fake backend (CPU),
and on the GPU each request's result alone and in the mix."""
import numpy as np
import pytest

from paper_1901_08140_gb300 import serving as S


class FakeBackend:
    """Completes a launch a fixed number of polls after it starts."""

    def __init__(self, slots=3, polls=5):
        self._slots = slots
        self.polls = polls
        self.log = []

    @property
    def slots(self):
        return self._slots

    def launch(self, req, slot):
        self.log.append(("launch", req.rid, slot))
        return {"req": req, "left": self.polls}

    def poll(self, h):
        h["left"] -= 1
        if h["left"] > 0:
            return None
        return {"n_real": h["req"].n_electrons, "status": 0}

    def release(self, h):
        self.log.append(("release", h["req"].rid))


class FakeGroupBackend(FakeBackend):
    def launch_group(self, reqs, slot):
        self.log.append(("group", tuple(r.rid for r in reqs), slot))
        return {"reqs": list(reqs), "left": self.polls}

    def poll_group(self, h):
        h["left"] -= 1
        if h["left"] > 0:
            return None
        return [{"n_real": r.n_electrons, "status": 0} for r in h["reqs"]]

    def release_group(self, h):
        self.log.append(("release", tuple(r.rid for r in h["reqs"])))


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3
        return self.t


def _reqs(sizes, arrivals):
    return [S.Request(i, None, None, arrival=a, n_electrons=n) for i, (n, a) in enumerate(zip(sizes, arrivals))]


def test_admission_respects_slots_and_budget():
    be = FakeBackend(slots=3)
    budget = S.BYTES_PER_ELECTRON * 2500 + 2 * S.BYTES_PER_SWARM
    srv = S.Server(be, memory_budget=budget, clock=Clock(), idle_sleep=0)
    done = srv.run(_reqs([1000, 1000, 1000, 500, 2000], [0, 0, 0, 0, 0]), realtime=False)
    assert sorted(r.rid for r in done) == [0, 1, 2, 3, 4]
    assert srv.max_concurrent <= 3
    assert srv.peak_in_use <= budget
    # admission is in arrival order: request 3 starts only after request 0 or 1 ends
    launches = [e for e in be.log if e[0] == "launch"]
    assert [e[1] for e in launches] == [0, 1, 2, 3, 4]
    assert all(r.done > r.admitted >= r.arrival for r in done)


def test_requests_arriving_while_others_run_are_admitted_at_once():
    be = FakeBackend(slots=4, polls=50)
    srv = S.Server(be, memory_budget=1e12, clock=Clock(), idle_sleep=0)
    done = srv.run(_reqs([10, 10, 10], [0.0, 0.005, 0.010]), realtime=True)
    by = {r.rid: r for r in done}
    # the later requests start before the first one finished
    assert by[1].admitted < by[0].done and by[2].admitted < by[0].done
    assert srv.max_concurrent == 3


def test_queued_requests_are_launched_together_within_budget():
    be = FakeGroupBackend(slots=2, polls=20)
    budget = S.BYTES_PER_ELECTRON * 3000 + 3 * S.BYTES_PER_SWARM
    srv = S.Server(be, memory_budget=budget, clock=Clock(), idle_sleep=0, max_group=8)
    done = srv.run(_reqs([1000] * 7, [0.0] * 7), realtime=False)
    groups = [e[1] for e in be.log if e[0] == "group"]
    assert groups[0] == (0, 1, 2)              # as many as the memory budget allows
    assert sorted(r for g in groups for r in g) == list(range(7))
    assert srv.peak_in_use <= budget and len(done) == 7


class FakeAloneBackend(FakeGroupBackend):
    """Requests with cfg == "alone" must be launched on their own."""

    @staticmethod
    def alone(req):
        return req.cfg == "alone"


def test_requests_that_run_alone_are_not_grouped():
    be = FakeAloneBackend(slots=2, polls=10)
    reqs = _reqs([100] * 6, [0.0] * 6)
    reqs[2].cfg = "alone"
    reqs[3].cfg = "alone"
    srv = S.Server(be, memory_budget=1e12, clock=Clock(), idle_sleep=0, max_group=8)
    done = srv.run(reqs, realtime=False)
    groups = [e[1] for e in be.log if e[0] == "group"]
    assert groups[:2] == [(0, 1), (2,)]
    assert (3,) in groups and sorted(r for g in groups for r in g) == list(range(6))
    assert len(done) == 6


def test_groups_hold_one_kernel_instance():
    class KeyBackend(FakeGroupBackend):
        @staticmethod
        def group_key(req):
            return req.cfg

    be = KeyBackend(slots=1, polls=3)
    reqs = _reqs([100] * 6, [0.0] * 6)
    for r, k in zip(reqs, [0, 0, 1, 1, 0, 1]):
        r.cfg = k
    srv = S.Server(be, memory_budget=1e12, clock=Clock(), idle_sleep=0, max_group=8)
    srv.run(reqs, realtime=False)
    groups = [e[1] for e in be.log if e[0] == "group"]
    assert groups == [(0, 1), (2, 3), (4,), (5,)]


def test_spawn_requests_reserve_memory_for_the_population_cap():
    class Cfg:
        spawn, pop_cap = 1, 10 ** 6
    r = S.Request(0, None, Cfg(), n_electrons=1)
    assert r.device_bytes() == (S.BYTES_PER_ELECTRON + S.BYTES_PER_BIRTH) * 10 ** 6 + S.BYTES_PER_SWARM


def test_oversized_request_is_rejected():
    srv = S.Server(FakeBackend(), memory_budget=1e6, clock=Clock(), idle_sleep=0)
    with pytest.raises(ValueError):
        srv.run(_reqs([10 ** 7], [0.0]))


def test_poisson_arrivals_and_summary():
    a = S.poisson_arrivals(1000.0, 20000, seed=3)
    gaps = np.diff(a)
    assert abs(gaps.mean() - 1e-3) < 3e-5 and np.all(gaps > 0)
    rs = _reqs([1] * 3, [0.0, 0.1, 0.2])
    for r, d in zip(rs, [0.05, 0.2, 0.4]):
        r.done = d
        r.tallies = {"n_real": 10}
    s = S.latency_summary(rs)
    assert s["requests"] == 3 and abs(s["p50_ms"] - 100.0) < 1e-9


@pytest.mark.gpu
def test_results_are_the_same_alone_and_in_the_mix():
    from paper_1901_08140_gb300 import build as B
    B.build()
    from paper_1901_08140_gb300 import bz
    from paper_1901_08140_gb300 import workloads as W
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
    for backend, arrivals in ((S.GpuBackend(ctx, n_streams=8), [0.0] * len(cfgs)),
                              (S.GpuBatchBackend(ctx, n_streams=3), list(np.linspace(0.0, 0.02, len(cfgs))))):
        reqs = [S.Request(i, m, c, arrival=a, n_electrons=int(c.n_electrons))
                for i, (m, c, a) in enumerate(zip(mixes, cfgs, arrivals))]
        srv = S.Server(backend, memory_budget=60e9, max_group=6)
        done = srv.run(reqs, realtime=True)
        assert srv.max_concurrent > 1 and len(done) == len(reqs)
        for r in done:
            a = alone[r.rid]
            for k in ("W", "eps", "D_L", "D_T", "n_real", "n_null", "n_window"):
                assert r.tallies[k] == a[k], (r.rid, k)


@pytest.mark.gpu
def test_avalanche_requests_alone_and_in_the_mix():
    """Spawn-mode requests run on worker threads beside batched swarms; the
    population they reach (integer counts, fixed by the ids' random numbers)
    is the same as when each runs alone."""
    from paper_1901_08140_gb300 import build as B
    B.build()
    from paper_1901_08140_gb300 import bz
    from paper_1901_08140_gb300 import workloads as W
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
    srv = S.Server(S.GpuBatchBackend(ctx, n_streams=3), memory_budget=60e9, max_group=4)
    done = srv.run(reqs, realtime=True)
    assert len(done) == len(reqs)
    for r in done:
        a = alone[r.rid]
        for k in ("n_particles", "n_real", "n_ion", "n_att", "n_spawned", "n_alive", "n_capped"):
            assert r.tallies[k] == a[k], (r.rid, k)
        assert r.tallies["eps"] == pytest.approx(a["eps"], rel=1e-12, abs=0.0)
