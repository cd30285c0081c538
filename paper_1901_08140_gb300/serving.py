"""Serving loop: swarm requests with continuous batching on one GPU.

Requests (a compiled mixture plus a swarm configuration) arrive over time.
Whenever a launch slot (one of S CUDA streams) is free, the server takes
the queued requests in arrival order, as many as fit the device-memory
admission budget (and a group-size cap), and launches them together as one
batched persistent launch on that slot; it polls completions without
blocking.  Groups on different slots run concurrently, so requests that
arrive while others are on the GPU are admitted as soon as a slot and
memory free up and their work overlaps on the device.  Each swarm's
results depend only on its configuration (counter-based random numbers
keyed by the swarm seed and particle ids, one step kernel for every launch
form), so a request's tallies are the same alone and in the mix.

The scheduling logic is independent of the GPU: a backend object launches,
polls and releases swarms (``GpuBackend`` drives libbz.so; the tests drive
the same server with a host-only fake to check admission and ordering).
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Callable, Deque, Dict, List, Optional, Sequence

import numpy as np

# device bytes per electron of a swarm (results in SoA) and per swarm (tally scratch)
BYTES_PER_ELECTRON = 92
BYTES_PER_SWARM = 2 << 20
BYTES_PER_BIRTH = 40   # spawn mode: birth record of a created electron


@dataclasses.dataclass
class Request:
    rid: int
    mixture: object                 # a compiled mixture (bz.Mixture) or backend-specific handle
    cfg: object                     # bz.bz_swarm_config
    arrival: float = 0.0            # seconds after the start of the run
    n_electrons: int = 0
    admitted: Optional[float] = None
    done: Optional[float] = None
    tallies: Optional[Dict[str, float]] = None
    status: int = 0

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    def device_bytes(self) -> int:
        cap = int(getattr(self.cfg, "pop_cap", 0) or 0) if getattr(self.cfg, "spawn", 0) else 0
        n = max(self.n_electrons, cap)
        return (BYTES_PER_ELECTRON + (BYTES_PER_BIRTH if cap else 0)) * n + BYTES_PER_SWARM


class GpuBackend:
    """Launches requests as swarms of libbz.so on a pool of CUDA streams."""

    def __init__(self, ctx, n_streams: int = 16):
        import torch
        from . import bz
        self.bz = bz
        self.ctx = ctx
        dev = torch.device("cuda", ctx.device)
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(n_streams)]

    @property
    def slots(self) -> int:
        return len(self.streams)

    def launch(self, req: Request, slot: int):
        return self.bz.Swarm(self.ctx, req.mixture, req.cfg, self.streams[slot])

    def poll(self, handle) -> Optional[Dict[str, float]]:
        t = self.bz.bz_tallies()
        import ctypes as C
        st = self.bz.lib().bz_query_tallies(handle.h, C.byref(t))
        if st == self.bz.BZ_ENOTREADY:
            return None
        out = self.bz._tally_dict(t)
        out["status"] = st
        return out

    def release(self, handle) -> None:
        handle.close()


class _SwarmRun:
    """A request launched on its own as a swarm (spawn mode: an avalanche)."""

    def __init__(self, bz, ctx, req, stream):
        self.bz = bz
        self.sw = bz.Swarm(ctx, req.mixture, req.cfg, stream)

    def poll(self) -> Optional[List[Dict[str, float]]]:
        import ctypes as C
        t = self.bz.bz_tallies()
        st = self.bz.lib().bz_query_tallies(self.sw.h, C.byref(t))
        if st == self.bz.BZ_ENOTREADY:
            return None
        out = self.bz._tally_dict(t)
        out["status"] = st
        return [out]

    def close(self) -> None:
        self.sw.close()


class GpuBatchBackend:
    """Launches groups of requests as one batched launch of libbz.so per slot;
    spawn-mode requests (avalanches) run alone, each in its own persistent
    launch on the slot's stream."""

    def __init__(self, ctx, n_streams: int = 4):
        import torch
        from . import bz
        self.bz = bz
        self.ctx = ctx
        dev = torch.device("cuda", ctx.device)
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(n_streams)]

    @property
    def slots(self) -> int:
        return len(self.streams)

    @staticmethod
    def alone(req: Request) -> bool:
        return bool(getattr(req.cfg, "spawn", 0))

    @staticmethod
    def group_key(req: Request):
        """Requests share a launch only with requests that run the same build
        of the step kernel alone, so that every result is the one the
        request gets alone: the feature build (the paper's adaptive trial
        frequencies, xi-form gases, moving targets) or the lean one, and in
        the lean one with or without a magnetic field."""
        info = getattr(req.mixture, "info", None) or {}
        ext = (getattr(req.cfg, "trial_mode", 0) in (3, 4) or info.get("n_xi_gases", 0) > 0
               or getattr(req.cfg, "gas_temperature_K", 0.0) > 0.0)
        return (bool(ext), bool(ext or getattr(req.cfg, "b_T", 0.0) > 0.0))

    def launch_group(self, reqs: Sequence[Request], slot: int):
        if len(reqs) == 1 and self.alone(reqs[0]):
            return _SwarmRun(self.bz, self.ctx, reqs[0], self.streams[slot])
        b = self.bz.Batch(self.ctx, [r.mixture for r in reqs], [r.cfg for r in reqs], use_graph=False)
        b.launch(self.streams[slot])
        return b

    def poll_group(self, handle) -> Optional[List[Dict[str, float]]]:
        if isinstance(handle, _SwarmRun):
            return handle.poll()
        if not handle.ready():
            return None
        return handle.tallies(check=False)

    def release_group(self, handle) -> None:
        handle.close()


class Server:
    """Continuous-batching request loop with memory-budget admission.

    With a backend that launches groups (``launch_group``), each free slot
    takes up to ``max_group`` queued requests at once; otherwise one request
    per slot.
    """

    def __init__(self, backend, memory_budget: float = 60e9, clock: Callable[[], float] = time.perf_counter,
                 idle_sleep: float = 2e-5, max_group: int = 512):
        self.backend = backend
        self.budget = float(memory_budget)
        self.clock = clock
        self.idle_sleep = idle_sleep
        self.max_group = max_group if hasattr(backend, "launch_group") else 1
        self.in_use = 0.0
        self.peak_in_use = 0.0
        self.max_concurrent = 0
        self.groups = 0

    def run(self, requests: Sequence[Request], realtime: bool = True) -> List[Request]:
        """Serves `requests` (sorted by arrival); returns them completed.

        With realtime=True a request becomes visible at its arrival time on
        the wall clock; otherwise all are visible at once (throughput mode).
        """
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in reqs:
            if r.device_bytes() > self.budget:
                raise ValueError(f"request {r.rid} needs {r.device_bytes()} bytes, above the admission budget")
        pending: Deque[Request] = collections.deque(reqs)
        queue: Deque[Request] = collections.deque()
        free = list(range(self.backend.slots))[::-1]
        running: Dict[int, tuple] = {}   # slot -> (requests, handle)
        t0 = self.clock()
        done: List[Request] = []
        grouped = self.max_group > 1
        while pending or queue or running:
            now = self.clock() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                queue.append(pending.popleft())
            # admit in arrival order while a slot and memory are free
            while queue and free and self.in_use + queue[0].device_bytes() <= self.budget:
                group, need = [], 0.0
                alone = getattr(self.backend, "alone", lambda r: False)
                key = getattr(self.backend, "group_key", lambda r: 0)
                while (queue and len(group) < self.max_group
                       and self.in_use + need + queue[0].device_bytes() <= self.budget):
                    if group and (alone(queue[0]) or key(queue[0]) != key(group[0])):
                        break          # runs on its own, or in another kernel instance
                    r = queue.popleft()
                    need += r.device_bytes()
                    group.append(r)
                    if alone(r):
                        break
                slot = free.pop()
                t_adm = self.clock() - t0
                for r in group:
                    r.admitted = t_adm
                h = self.backend.launch_group(group, slot) if grouped else self.backend.launch(group[0], slot)
                running[slot] = (group, h)
                self.groups += 1
                self.in_use += need
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                self.max_concurrent = max(self.max_concurrent, sum(len(g) for g, _ in running.values()))
            progressed = False
            for slot in list(running):
                group, h = running[slot]
                res = self.backend.poll_group(h) if grouped else self.backend.poll(h)
                if res is None:
                    continue
                t_done = self.clock() - t0
                if not grouped:
                    res = [res]
                for r, t in zip(group, res):
                    r.done = t_done
                    r.tallies = t
                    r.status = int(t.get("status", 0))
                    self.in_use -= r.device_bytes()
                    done.append(r)
                (self.backend.release_group if grouped else self.backend.release)(h)
                del running[slot]
                free.append(slot)
                progressed = True
            if not progressed and self.idle_sleep > 0:
                time.sleep(self.idle_sleep)
        return done


def poisson_arrivals(rate: float, count: int, seed: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def latency_summary(done: Sequence[Request], duration: Optional[float] = None) -> Dict[str, float]:
    lat = np.array([r.latency for r in done])
    reals = sum(int(r.tallies["n_real"]) for r in done if r.tallies)
    span = duration if duration is not None else max(r.done for r in done) - min(r.arrival for r in done)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "real_collisions_per_s": reals / span if span > 0 else math.nan, "span_s": span}
