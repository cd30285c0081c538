"""Serving: swarm requests with continuous batching on one GPU.

The request loop itself is native (``bz_server_*``, ``bz_submit``,
``bz_poll``, ``bz_cancel`` in libbz.so): a worker thread admits queued
requests in arrival order into free launch slots as device memory allows,
batches requests of one step-kernel class into one persistent launch per
slot, runs avalanche (spawn-mode) requests alone, and polls completions
without blocking.  This module only marshals: ``Server.run`` submits each
request at its arrival time and collects the results with the server's own
timestamps.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import bz


@dataclasses.dataclass
class Request:
    rid: int
    mixture: object                 # a compiled mixture (bz.Mixture), or None on a simulated server
    cfg: object                     # bz.bz_swarm_config
    arrival: float = 0.0            # seconds after the start of the run
    n_electrons: int = 0
    submitted: Optional[float] = None  # when the loop handed it to the server (>= arrival)
    admitted: Optional[float] = None
    done: Optional[float] = None
    tallies: Optional[Dict[str, float]] = None
    status: int = 0
    launch: int = -1
    group_size: int = 0

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Server:
    """A bz_server: continuous-batching request loop of libbz.so.

    simulate = n > 0 runs the scheduling on the host only (no device; a launch
    ends after n polls of the worker), for tests on machines without a GPU.
    """

    def __init__(self, ctx=None, memory_budget: float = 60e9, n_slots: int = 3, max_group: int = 512,
                 simulate: int = 0):
        # the server's worker thread allocates every launch's memory; it does
        # so through a context of its own on the same device that uses CUDA's
        # stream-ordered allocator, so a native thread never calls back into
        # Python (mixtures of any context on that device may be submitted)
        self.ctx = bz.Context(ctx.device, torch_allocator=False) if ctx is not None and not simulate else None
        opts = bz.bz_server_opts(float(memory_budget), int(n_slots), int(max_group), int(simulate), 0)
        h = C.c_void_p()
        bz._check(bz.lib().bz_server_create(self.ctx.h if self.ctx is not None else None, C.byref(opts),
                                            C.byref(h)))
        self.h = h

    def submit(self, mixture, cfg) -> int:
        rid = C.c_uint64()
        bz._check(bz.lib().bz_submit(self.h, mixture.h if mixture is not None else None, C.byref(cfg),
                                     C.byref(rid)))
        return int(rid.value)

    def poll(self, rid: int):
        """None while queued or running; else (status, tallies, info)."""
        t, info = bz.bz_tallies(), bz.bz_request_info()
        st = bz.lib().bz_poll(self.h, C.c_uint64(rid), C.byref(t), C.byref(info))
        if st == bz.BZ_ENOTREADY:
            return None
        if st == bz.BZ_EINVAL:
            bz._check(st)
        out = bz._tally_dict(t)
        out["status"] = st
        return st, out, {k: getattr(info, k) for k, _ in bz.bz_request_info._fields_}

    def pause(self, paused: bool = True) -> None:
        """Holds (or resumes) admission; running launches go on."""
        bz._check(bz.lib().bz_server_pause(self.h, int(bool(paused))))

    def cancel(self, rid: int) -> None:
        bz._check(bz.lib().bz_cancel(self.h, C.c_uint64(rid)))

    def stats(self) -> Dict[str, float]:
        s = bz.bz_server_stats()
        bz._check(bz.lib().bz_server_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in bz.bz_server_stats._fields_}

    def run(self, requests: Sequence[Request], realtime: bool = True, poll_sleep: float = 2e-5) -> List[Request]:
        """Submits `requests` at their arrival times (all at once when
        realtime is False) and returns them completed.  A request's admission
        and completion are the server's times after its submission, added to
        the moment this loop submitted it, so a latency (completion minus
        arrival) includes any delay of the loop in submitting."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        if not reqs:
            return []
        t0 = time.perf_counter()
        waiting: Dict[int, Request] = {}
        done: List[Request] = []
        i = 0
        while i < len(reqs) or waiting:
            now = time.perf_counter() - t0
            while i < len(reqs) and (not realtime or reqs[i].arrival <= now):
                r = reqs[i]
                waiting[self.submit(r.mixture, r.cfg)] = r
                r.submitted = max(time.perf_counter() - t0, r.arrival) if realtime else r.arrival
                i += 1
            for rid in list(waiting):
                res = self.poll(rid)
                if res is None:
                    continue
                st, t, info = res
                r = waiting.pop(rid)
                # the server's clock from submission on, this loop's before
                r.status, r.tallies = int(st), t
                r.admitted = r.submitted + (info["t_admit"] - info["t_submit"])
                r.done = r.submitted + (info["t_done"] - info["t_submit"])
                r.launch, r.group_size = int(info["launch"]), int(info["group_size"])
                done.append(r)
            if waiting and poll_sleep > 0:
                time.sleep(poll_sleep)
        return done

    def close(self):
        if getattr(self, "h", None):
            bz.lib().bz_server_destroy(self.h)
            self.h = None
        if getattr(self, "ctx", None) is not None:
            self.ctx.close()
            self.ctx = None

    def __del__(self):
        import sys
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def poisson_arrivals(rate: float, count: int, seed: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def latency_summary(done: Sequence[Request], duration: Optional[float] = None) -> Dict[str, float]:
    lat = np.array([r.latency for r in done])
    reals = sum(int(r.tallies["n_real"]) for r in done if r.tallies)
    span = duration if duration is not None else max(r.done for r in done) - min(r.arrival for r in done)
    lag = np.array([(r.submitted if r.submitted is not None else r.arrival) - r.arrival for r in done])
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "real_collisions_per_s": reals / span if span > 0 else math.nan, "span_s": span,
            "submit_lag_p99_ms": float(np.percentile(lag, 99) * 1e3), "submit_lag_max_ms": float(lag.max() * 1e3)}
