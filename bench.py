#!/usr/bin/env python
"""Benchmark of the electron-swarm step loop on GB300.

One step = the whole hot path over one batch: the Argon-like E/N sweep
(32 log-spaced points, 1-1000 Td), 1e6 electrons per point, each electron
run to its 1000th real collision with FP32 flights and FP64 tallies, every
swarm's tallies reduced on the device and copied to the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``value`` is real collisions per second over
all ranks (device time, CUDA events on the launching stream, max over
ranks); ``e2e`` is the same metric through the C ABI with host tables and a
host read of the tallies inside the timed region; ``roofline`` relates the
step kernel's algorithmic thread operations to the SM issue rate;
``cpu_baseline`` is the FP64 oracle timed on this host's cores.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "collisions/s batched vs plain at ≤0.5% drift-velocity error; p99 swarm latency"
UNIT = "real collisions/s"
# Algorithmic thread operations of one trial step and the extra of a real
# collision (counted from the method's arithmetic; see the design notes).
ALG_OPS_PER_TRIAL = 95
ALG_OPS_PER_REAL = 90
SM_COUNT_NOMINAL = 152
LANES_PER_SM_CLOCK = 4 * 32     # 4 schedulers x 32 lanes issue per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--points", type=int, default=32)
    ap.add_argument("--electrons", type=int, default=1_000_000)
    ap.add_argument("--collisions", type=int, default=1000)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="bound of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--only-point", type=int, default=-1, help="run one E/N point of the sweep (profiling case)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-rates", default="250,1000,2000", help="Poisson arrival rates [req/s] of the serving run")
    ap.add_argument("--serve-seconds", type=float, default=1.0, help="arrival window of each serving run")
    ap.add_argument("--avalanche-cap", type=int, default=100_000,
                    help="population cap of the serving run's avalanche requests")
    ap.add_argument("--avalanche-frac", type=float, default=0.05, help="fraction of avalanche requests")
    ap.add_argument("--no-strategies", action="store_true", help="skip the trial-frequency comparison")
    ap.add_argument("--no-batched-workload", action="store_true", help="skip the 256-swarm batched workload")
    ap.add_argument("--strategy-electrons", type=int, default=100_000)
    ap.add_argument("--trial", choices=["window", "lazy"], default="window",
                    help="trial frequency: exact windowed local bound (default) or the constant maximum")
    return ap.parse_args()


def dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def profiled_traffic():
    """DRAM bytes (read + write) of one batched step-kernel launch of this
    workload from an ncu capture, if the kernel sources are still the ones
    that capture ran; None otherwise."""
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    try:
        with open(os.path.join(root, "profiles", "batch_kernel_traffic_argon_sweep.json")) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for name in rec["sources"]:
            with open(os.path.join(root, "paper_1901_08140_gb300", "csrc", name), "rb") as f:
                h.update(f.read())
    except (OSError, ValueError, KeyError):
        return None
    if h.hexdigest() != rec["sources_sha256"]:
        return None
    return rec["dram_bytes_read"] + rec["dram_bytes_write"]


def workload_name(args):
    """The workload both arms name in their JSON line (the same swarms; how
    each arm samples them is in its own keys)."""
    return (f"Argon-like E/N sweep: {args.points} log points 1-1000 Td x {args.electrons} electrons x "
            f"{args.collisions} real collisions, FP32 flights, FP64 tallies, {args.trial} trial frequency, B = 0"
            + (f" (point {args.only_point} only)" if args.only_point >= 0 else ""))


def sweep_specs(args, rank):
    from paper_1901_08140_gb300 import workloads as W
    specs = W.argon_sweep(n_electrons=args.electrons, real_collisions=args.collisions, points=args.points)
    if args.only_point >= 0:
        specs = [specs[args.only_point]]
    return specs


def cpu_baseline(args, specs, budget_s):
    """The FP64 oracle, as it stands, on this host's cores: a bounded sample
    of the same sweep (the same particle ids of each point, taken point by
    point in a round-robin of id blocks until the time bound)."""
    from oracle import oracle as O
    m = O.Mixture(specs[0].gases)
    cores = O.cpu_count()
    block = 64 * cores
    reals = trials = 0
    t0 = time.perf_counter()
    rounds = 0
    done_points = 0
    while True:
        for i, s in enumerate(specs):
            p = O.run_swarm(m, e_over_n_Td=s.e_over_n_Td, real_collisions=s.real_collisions, n=block, seed=s.seed,
                            id0=rounds * block, threads=cores)
            reals += int(p["n_real"].sum())
            trials += int(p["n_real"].sum() + p["n_null"].sum() + p["n_fail"].sum())
            done_points += 1
            if time.perf_counter() - t0 > budget_s and done_points >= min(len(specs), 4):
                break
        else:
            rounds += 1
            continue
        break
    dt = time.perf_counter() - t0
    sample = (f"{done_points} (E/N point, {block}-electron id block) units of the sweep, "
              f"I={specs[0].real_collisions}, {reals} real / {trials} trial collisions in {dt:.1f} s")
    return {"value": reals / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "trial_collisions_per_s": trials / dt}


def _timed(stream, flush, steps, fn, world, dev):
    """Runs fn() `steps` times; device time per step from CUDA events on `stream`."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    outs = []
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        ev0.record(stream)
        h = fn()
        ev1.record(stream)
        ev1.synchronize()
        total += ev0.elapsed_time(ev1)
        torch.cuda.synchronize(dev)
        outs.append(h)
    return total, outs


def batched_workload_runs(ctx, stream, flush, world, dev, collisions, warmup, steps):
    """The batched workload: 256 swarms, electrons log-uniform 1e3-1e6, 2-4
    of 8 synthetic gases each with Dirichlet fractions, E/N log-uniform
    0.1-1000 Td, |B| uniform 0-2 T at a random angle, I real collisions,
    windowed trial frequency.  Plain: one persistent launch per swarm, back
    to back; batched: all swarms in one persistent launch replayed from a
    CUDA graph with the autotuner's launch options."""
    from paper_1901_08140_gb300 import autotune, bz
    from paper_1901_08140_gb300 import workloads as W
    specs = W.batched_swarms(count=256, real_collisions=collisions)
    mixes = [bz.Mixture(ctx, s.gases) for s in specs]
    cfgs = [bz.config_from_spec(s, trial_mode=bz.BZ_TRIAL_WINDOW) for s in specs]

    def plain_step():
        return [bz.run_swarm(ctx, m, c, stream) for m, c in zip(mixes, cfgs)]

    for _ in range(warmup):
        for sw in plain_step():
            sw.tallies(check=False)
            sw.close()
    plain_ms, outs = _timed(stream, flush, steps, plain_step, world, dev)
    plain_reals = 0
    for sws in outs:
        for sw in sws:
            plain_reals += sw.tallies(check=False)["n_real"]
            sw.close()
    choice = autotune.tune(ctx, mixes, cfgs)
    batch = bz.Batch(ctx, mixes, autotune.apply(cfgs, choice), tile_particles=choice["tile_particles"],
                     blocks_per_sm=choice["blocks_per_sm"])
    for _ in range(warmup):
        batch.launch(stream)
        batch.tallies(check=False)
    ms = 0.0
    reals = 0
    for _ in range(steps):
        m1, _ = _timed(stream, flush, 1, lambda: batch.launch(stream), world, dev)
        ms += m1
        reals += sum(t["n_real"] for t in batch.tallies(check=False))
    batch.close()
    value, plain_value = reals / (ms / 1e3), plain_reals / (plain_ms / 1e3)
    return {"workload": "256 swarms, 1e3-1e6 electrons (log-uniform, %d in all), 2-4 of 8 synthetic gases, "
                        "E/N 0.1-1000 Td, |B| 0-2 T at random angles, I = %d" % (sum(c.n_electrons for c in cfgs),
                                                                                  collisions),
            "value": value, "unit": UNIT, "ms_per_step": ms / steps, "plain": {"value": plain_value,
            "ms_per_step": plain_ms / steps}, "batched_over_plain": value / plain_value,
            "autotuned": {k: choice[k] for k in ("window_c", "tile_particles", "blocks_per_sm", "cached")}}


def strategy_runs(ctx, mix, specs, electrons):
    """The argon sweep at `electrons` per point under each trial frequency
    (Sec. 6): real collisions/s of the step kernel, efficiency (Eq. 28),
    fails, electrons stopped by an error, and the largest deviation of W
    from the exact windowed run in combined standard errors."""
    import math
    from paper_1901_08140_gb300 import bz
    modes = [("window", bz.BZ_TRIAL_WINDOW), ("lazy", bz.BZ_TRIAL_LAZY), ("variable", bz.BZ_TRIAL_VARIABLE),
             ("binned", bz.BZ_TRIAL_BINNED)]
    out, ref = {}, None
    for name, mode in modes:
        cfgs = [bz.config_from_spec(s, n_electrons=electrons, trial_mode=mode, zeta=0.25, grace=5000,
                                    bins_per_decade=8, max_trials=10 ** 7) for s in specs]
        b = bz.Batch(ctx, [mix] * len(cfgs), cfgs, use_graph=False)
        b.launch()
        b.tallies(check=False)
        b.launch()
        ts = b.tallies(check=False)
        ms, _ = b.timing()
        b.close()
        reals = sum(t["n_real"] for t in ts)
        trials = sum(t["n_real"] + t["n_null"] + t["n_fail"] for t in ts)
        row = {"real_collisions_per_s": reals / (ms / 1e3), "efficiency": reals / trials if trials else None,
               "fails": int(sum(t["n_fail"] for t in ts)), "stopped_by_error": int(sum(t["n_incomplete"] for t in ts))}
        if ref is None:
            ref = ts
        else:
            z = [abs(t["W"] - r["W"]) / math.hypot(t["W_se"], r["W_se"]) for t, r in zip(ts, ref)
                 if t["W_se"] > 0 and r["W_se"] > 0]
            row["max_z_W_vs_window"] = max(z) if z else None
        out[name] = row
    return {"electrons_per_point": electrons, "zeta": 0.25, "grace": 5000, "bins_per_decade": 8, "modes": out}


def serving_runs(ctx, rates, seconds, collisions=100, pool=64, streams=3, avalanche_frac=0.05,
                 avalanche_cap=100_000):
    """Continuous-batching request loop under Poisson arrivals: swarm sizes,
    mixtures and fields of the batched workload (a pool of compiled
    mixtures), I real collisions per request, windowed trial frequency; a
    fraction are avalanche requests (Ar/CO2 93/7, 300 Td, spawn mode, one
    seed electron, 1 ns, population cap avalanche_cap)."""
    from paper_1901_08140_gb300 import bz, serving
    from paper_1901_08140_gb300 import workloads as W
    import numpy as np
    specs = W.batched_swarms(count=pool, real_collisions=collisions)
    mixes = [bz.Mixture(ctx, s.gases) for s in specs]
    ava_mix = bz.Mixture(ctx, W.ar_co2_avalanche_mixture())
    backend = serving.GpuBatchBackend(ctx, n_streams=streams)
    out = []
    for k, rate in enumerate(rates):
        n = max(1, int(rate * seconds))
        arr = serving.poisson_arrivals(rate, n, seed=100 + k)
        rng = np.random.default_rng(200 + k)
        reqs = []
        for i in range(n):
            seed = W.swarm_seed(10 ** 6 + 10 ** 4 * k + i)
            if rng.uniform() < avalanche_frac:
                cfg = bz.make_config(n_electrons=1, real_collisions=10 ** 9, e_over_n_Td=300.0, seed=seed,
                                     t_end_s=1e-9, spawn=True, pop_cap=avalanche_cap,
                                     trial_mode=bz.BZ_TRIAL_WINDOW)
                reqs.append(serving.Request(i, ava_mix, cfg, arrival=float(arr[i]), n_electrons=1))
                continue
            j = int(rng.integers(pool))
            cfg = bz.config_from_spec(specs[j], trial_mode=bz.BZ_TRIAL_WINDOW, seed=seed)
            reqs.append(serving.Request(i, mixes[j], cfg, arrival=float(arr[i]), n_electrons=int(cfg.n_electrons)))
        srv = serving.Server(backend, memory_budget=60e9)
        done = srv.run(reqs, realtime=True)
        summ = serving.latency_summary(done)
        ava = [r for r in done if getattr(r.cfg, "spawn", 0)]
        plain = [r for r in done if not getattr(r.cfg, "spawn", 0)]
        offered = sum(r.n_electrons for r in plain) * collisions / arr[-1] if n > 1 else float("nan")
        if ava:
            summ["avalanche"] = {"requests": len(ava),
                                 "p99_ms": float(np.percentile([r.latency for r in ava], 99) * 1e3),
                                 "mean_final_population": float(np.mean([r.tallies["n_particles"] for r in ava]))}
        offered += sum(r.tallies["n_real"] for r in ava) / arr[-1] if n > 1 else 0.0
        summ.update({"rate_req_s": rate, "offered_real_collisions_per_s": offered,
                     "max_concurrent": srv.max_concurrent, "launch_groups": srv.groups})
        out.append(summ)
    return out


def run_ours(args):
    import torch
    world, rank, local = dist()
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1901_08140_gb300 import build as B
    B.build()
    from paper_1901_08140_gb300 import bz
    specs = sweep_specs(args, rank)
    ctx = bz.Context(local)
    mix = bz.Mixture(ctx, specs[0].gases)
    # weak scaling: every rank runs the whole sweep on its own particle ids
    mode = bz.BZ_TRIAL_WINDOW if args.trial == "window" else bz.BZ_TRIAL_LAZY
    from paper_1901_08140_gb300 import sharding
    cfgs = [bz.config_from_spec(s, id_offset=sharding.weak_offset(rank, args.electrons), trial_mode=mode)
            for s in specs]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    # ---- plain: one persistent launch per swarm, back to back on one stream
    def plain_step():
        return [bz.run_swarm(ctx, mix, c, stream) for c in cfgs]

    for _ in range(args.warmup):
        for sw in plain_step():
            sw.tallies()
            sw.close()
    plain_ms, plain_outs = _timed(stream, flush, args.steps, plain_step, world, dev)
    plain_reals = 0
    for sws in plain_outs:
        for sw in sws:
            plain_reals += sw.tallies()["n_real"]
            sw.close()

    # ---- batched: every swarm in one persistent launch, replayed from a CUDA graph,
    # with the launch options the autotuner picks (cached per GPU and workload class)
    from paper_1901_08140_gb300 import autotune
    choice = autotune.tune(ctx, [mix] * len(cfgs), cfgs)
    bcfgs = autotune.apply(cfgs, choice)
    batch = bz.Batch(ctx, [mix] * len(cfgs), bcfgs, tile_particles=choice["tile_particles"],
                     blocks_per_sm=choice["blocks_per_sm"])

    def batch_step():
        batch.launch(stream)
        return None

    for _ in range(args.warmup):
        batch_step()
        batch.tallies()
    clocks = Clocks(local)
    reals = trials = 0
    kern_ms = 0.0
    steps_other = 0
    work = 0.0
    w_err = []
    total_ms = 0.0
    for _ in range(args.steps):
        ms, _ = _timed(stream, flush, 1, batch_step, world, dev)
        total_ms += ms
        ts = batch.tallies()
        km, _ = batch.timing()
        kern_ms += km
        for t in ts:
            tr = t["n_real"] + t["n_null"] + t["n_fail"]
            reals += t["n_real"]
            trials += tr
            steps_other += t["n_window"]
            work += ALG_OPS_PER_TRIAL * (tr + t["n_window"]) + ALG_OPS_PER_REAL * t["n_real"]
            w_err.append(t["W_se"] / abs(t["W"]) if t["W"] else float("inf"))
    clk = clocks.stop()
    launches = 5 * args.steps   # batch kernel + 4 multi-swarm tally kernels, in one graph
    t_max, tot_reals = sharding.reduce_step(total_ms, reals)
    p_max, tot_plain = sharding.reduce_step(plain_ms, plain_reals)
    value = tot_reals / (t_max / 1e3)
    plain_value = tot_plain / (p_max / 1e3)

    # end to end through the C ABI: host tables in, host tallies out
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        m2 = bz.Mixture(ctx, specs[0].gases)
        b2 = bz.Batch(ctx, [m2] * len(cfgs), bcfgs, tile_particles=choice["tile_particles"],
                      blocks_per_sm=choice["blocks_per_sm"])
        b2.launch(stream)
        e_reals = sum(t["n_real"] for t in b2.tallies())
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        h2d = m2.info["table_bytes"] + len(cfgs) * (C.sizeof(bz.bz_swarm_config) + 4096)
        d2h = len(cfgs) * C.sizeof(bz.bz_tallies)
        b2.close()
        m2.close()
        e2e = {"value": e_reals / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    batch.close()

    sm_mhz = clk.get("sm_mhz") or 2070.0
    peak = torch.cuda.get_device_properties(dev).multi_processor_count * LANES_PER_SM_CLOCK * sm_mhz * 1e6
    achieved = work / (kern_ms / 1e3)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
                "frac": achieved / peak, "traffic": profiled_traffic(),
                "kernel": "batch_kernel (lean FP32 build without field paths; 4 blocks/SM where the tables fit)",
                "note": f"algorithmic thread-ops ({ALG_OPS_PER_TRIAL}/step + {ALG_OPS_PER_REAL}/real) over "
                        f"SMs x 128 lanes x median SM clock {sm_mhz:.0f} MHz"}
    batched_workload = None
    if not args.no_batched_workload and args.only_point < 0:
        batched_workload = batched_workload_runs(ctx, stream, flush, world, dev, args.collisions,
                                                 max(1, args.warmup - 2), max(1, min(args.steps, 2)))
    strategies = None
    if not args.no_strategies and rank == 0:
        strategies = strategy_runs(ctx, mix, specs, min(args.strategy_electrons, args.electrons))
    serve = None
    if not args.no_serving and rank == 0:
        rates = [float(x) for x in args.serve_rates.split(",") if x]
        serve = serving_runs(ctx, rates, args.serve_seconds, avalanche_frac=args.avalanche_frac,
                             avalanche_cap=args.avalanche_cap)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(args, specs, args.cpu_seconds)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(args),
                   "mode": "batched: all swarms in one persistent launch replayed from a CUDA graph",
                   "swarms": len(specs), "electrons_per_swarm": args.electrons, "real_collisions": args.collisions,
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"dp{world} (particle ids)",
                   "autotuned": {k: choice[k] for k in ("window_c", "tile_particles", "blocks_per_sm", "cached")}},
        "plain": {"value": plain_value, "ms_per_step": p_max / args.steps,
                  "mode": "one persistent launch per swarm, back to back on one stream"},
        "batched_over_plain": value / plain_value,
        "trial_collisions_per_s": trials * world / (t_max / 1e3),
        "efficiency": reals / trials if trials else None,
        "window_restarts_per_real": steps_other / reals if reals else None,
        "max_rel_se_W": max(w_err) if w_err else None,
        "trial_frequency": args.trial,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
        "batched_workload": batched_workload,
        "trial_strategies": strategies,
        "serving": serve,
        # p99 at the highest arrival rate the GPU kept up with (>= 90 % of the offered work)
        "p99_swarm_latency_ms": (max(((x["rate_req_s"], x["p99_ms"]) for x in serve
                                      if x["real_collisions_per_s"] >= 0.9 * x["offered_real_collisions_per_s"]),
                                     default=(None, None))[1] if serve else None),
    }
    print(json.dumps(out), flush=True)


def run_reference(args):
    world, rank, local = dist()
    if rank != 0:
        return
    from oracle import oracle as O
    specs = sweep_specs(args, 0)
    m = O.Mixture(specs[0].gases)
    cores = O.cpu_count()
    block = 16 * cores
    # one step: a bounded sample of the sweep (every E/N point, `block` electrons)

    def step(k):
        r = t = 0
        for s in specs:
            p = O.run_swarm(m, e_over_n_Td=s.e_over_n_Td, real_collisions=s.real_collisions, n=block, seed=s.seed,
                            id0=k * block, threads=cores)
            r += int(p["n_real"].sum())
            t += int(p["n_real"].sum() + p["n_null"].sum() + p["n_fail"].sum())
        return r, t

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    reals = trials = 0
    for k in range(args.steps):
        r, t = step(args.warmup + k)
        reals += r
        trials += t
    dt = time.perf_counter() - t0
    value = reals / dt
    sample = (f"per step: all {len(specs)} E/N points x {block} electrons x I={specs[0].real_collisions} "
              f"(FP64 oracle, Lazy exact trial frequency, {cores} threads)")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": workload_name(args), "sample": sample},
        "trial_collisions_per_s": trials / dt,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
