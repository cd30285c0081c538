#!/usr/bin/env python
"""Benchmark of the electron-swarm step loop on GB300.

One step = the whole hot path over one batch: the batched workload of 256
swarms (1e3-1e6 electrons each, log-uniform, 4.1e7 in all; each a mixture
of 2-4 of 8 synthetic gases with 5-40 channels on 100-1000-point tables;
E/N log-uniform 0.1-1000 Td; |B| uniform 0-2 T at a random angle to E),
every electron run to its 1000th real collision with FP32 flights and FP64
tallies, all swarms in one persistent launch replayed from a CUDA graph,
every swarm's tallies reduced on the device and copied to the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``value`` is real collisions per second of
the batched launch over all ranks (device time, CUDA events on the
launching stream, max over ranks); ``plain`` is the same swarms launched
one by one at the same window length; ``e2e`` is the same metric through
the C ABI from host buffers (tables compiled and copied, configurations
copied, tallies read back) inside the timed region; ``roofline`` relates the
step kernel's algorithmic thread operations to the SM issue rate;
``cpu_baseline`` is the FP64 oracle timed on this host's cores.  Further
keys: four swarms of the batched workload against the oracle, the
Argon-like sweep (its throughput, its roofline and its drift velocity
against the oracle, the metric's accuracy qualifier), the Maxwell
and Ar/CO2 configurations, FP32 against FP64, the paper's trial
frequencies, and serving latency under Poisson load.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
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
SM_COUNT_NOMINAL = 152
LANES_PER_SM_CLOCK = 4 * 32     # 4 schedulers x 32 lanes issue per clock
# Algorithmic thread operations of the method, counted from its arithmetic
# (per trial step, per new trial-frequency window, per real collision) for
# the two kernel classes the workloads run: "plain" -- B = 0, a few
# channels searched in shared memory (the Argon-like sweep); "field" -- B != 0
# and many channels searched in global memory by a guided bisection of
# cumulative tables (the batched workload, Ar/CO2 with B).
ALG_OPS = {
    "plain": {"step": 95, "window": 61, "real": 67},
    "field": {"step": 128, "window": 86, "real": 135},
}
LEGS = ("plain", "e2e", "sweep", "oracle", "configs", "precision", "strategies", "avalanche", "serving", "cpu")
L2_NOTE = "flushed between steps (256 MiB write)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["batched", "sweep"], default="batched",
                    help="the headline workload (sweep: the Argon-like E/N sweep)")
    ap.add_argument("--swarms", type=int, default=256, help="swarms of the batched workload")
    ap.add_argument("--scale", type=int, default=1, help="divide every swarm's electrons by this (profiling case)")
    ap.add_argument("--collisions", type=int, default=1000)
    ap.add_argument("--points", type=int, default=32, help="E/N points of the sweep")
    ap.add_argument("--electrons", type=int, default=1_000_000, help="electrons per point of the sweep")
    ap.add_argument("--legs", default="all", help="comma list of " + ",".join(LEGS) + ", or all / none")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="bound of the CPU-baseline sample")
    ap.add_argument("--batched-oracle-electrons", type=int, default=32_000,
                    help="oracle electrons per swarm of the batched workload's check against the oracle")
    ap.add_argument("--oracle-electrons", type=int, default=10_000,
                    help="oracle electrons per E/N point of the sweep's drift-velocity check")
    ap.add_argument("--serve-rates", default="250,400,600,800,2000", help="Poisson arrival rates [req/s]")
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="arrival window of each serving run")
    ap.add_argument("--serve-rates-i1000", default="25,50,75,100",
                    help="Poisson arrival rates [req/s] of the serving sweep at I = 1000 real collisions per request")
    ap.add_argument("--serve-slots", type=int, default=3, help="launch slots (streams) of the serving loop")
    ap.add_argument("--serve-max-group", type=int, default=512, help="requests per launch at most")
    ap.add_argument("--avalanche-cap", type=int, default=100_000,
                    help="population cap of the serving run's avalanche requests")
    ap.add_argument("--avalanche-frac", type=float, default=0.05, help="fraction of avalanche requests")
    ap.add_argument("--avalanche-caps", default="1e5,1e7,1e8",
                    help="population caps of the avalanche leg (one seed electron each, run alone)")
    ap.add_argument("--strategy-electrons", type=int, default=100_000)
    ap.add_argument("--precision-electrons", type=int, default=100_000,
                    help="electrons per swarm of the FP32-against-FP64 comparison")
    ap.add_argument("--no-tune", action="store_true",
                    help="the autotuner's default launch options instead of a search (profiling runs)")
    ap.add_argument("--only-point", type=int, default=-1, help="sweep workload: one E/N point (profiling case)")
    ap.add_argument("--block-threads", type=int, default=0,
                    help="with --no-tune: threads per block of the headline launch (profiling runs)")
    ap.add_argument("--smem-budget", type=int, default=0,
                    help="with --no-tune: table budget per block the headline's mixtures are compiled for")
    a = ap.parse_args()
    a.legs = set(LEGS) if a.legs == "all" else set() if a.legs == "none" else set(a.legs.split(","))
    return a


def _jsonable(o):
    """numpy scalars and arrays as plain JSON values."""
    import numpy as np
    if isinstance(o, np.bool_):
        return bool(o)
    if isinstance(o, np.integer):
        return int(o)
    if isinstance(o, np.floating):
        return float(o)
    if isinstance(o, np.ndarray):
        return o.tolist()
    raise TypeError(f"{type(o).__name__} is not JSON serializable")


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


def _profile_record(name):
    """profiles/<name>.json if the kernel sources are still the ones its ncu
    capture ran (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", name + ".json")) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, "paper_1901_08140_gb300", "csrc", src), "rb") as f:
                h.update(f.read())
    except (OSError, ValueError, KeyError):
        return None
    return rec if h.hexdigest() == rec["sources_sha256"] else None


def _same_launch(rec, launch):
    """The captured launch had this block size and table budget."""
    base = {"block_threads": 256, "smem_budget": 0}
    return launch is None or all(int(rec.get("launch", {}).get(k, base[k])) == int(v or base[k])
                                 for k, v in launch.items())


def profiled_traffic(name, launch=None):
    """DRAM bytes (read + write) of one step-kernel launch of a workload from
    an ncu capture summarised in profiles/<name>.json, if the kernel sources
    are still the ones that capture ran and the capture launched the same
    block size and table budget (else None)."""
    rec = _profile_record(name)
    if rec is None or not _same_launch(rec, launch):
        return None
    return (rec["dram_bytes_read"] + rec["dram_bytes_write"]) * rec.get("scale_to_full", 1.0)


def shared_memory_roofline(case, reals, kern_ms, sm_count, sm_mhz, launch=None):
    """Shared-memory pipe use of a launch: shared-memory wavefronts per real
    collision from the ncu capture of the workload's reduced case
    (profiles/batch_kernel_smem.json, same launch form) times this launch's
    real collisions, over the peak of one 128-byte wavefront per SM per clock."""
    rec = _profile_record("batch_kernel_smem")
    if rec is None or case not in rec["cases"] or not _same_launch(rec["cases"][case], launch):
        return None
    per_real = rec["cases"][case]["wavefronts_per_real"]
    achieved = per_real * reals * 128.0 / (kern_ms / 1e3)
    peak = sm_count * 128.0 * sm_mhz * 1e6
    return {"achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TB/s", "frac": achieved / peak,
            "wavefronts_per_real": per_real, "source": rec["cases"][case]["command"]}


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def batched_specs(args):
    from paper_1901_08140_gb300 import workloads as W
    specs = W.batched_swarms(count=args.swarms, real_collisions=args.collisions)
    if args.scale > 1:
        import dataclasses
        specs = [dataclasses.replace(s, n_electrons=max(1, s.n_electrons // args.scale)) for s in specs]
    return specs


def sweep_specs(args):
    from paper_1901_08140_gb300 import workloads as W
    specs = W.argon_sweep(n_electrons=max(1, args.electrons // args.scale), real_collisions=args.collisions,
                          points=args.points)
    return [specs[args.only_point]] if args.only_point >= 0 else specs


def batched_name(args, specs):
    n = sum(s.n_electrons for s in specs)
    return (f"{len(specs)} swarms, electrons log-uniform 1e3-1e6 ({n} in all"
            + (f", each swarm's count divided by {args.scale}" if args.scale > 1 else "")
            + "), 2-4 of 8 synthetic gases (5-40 channels, 100-1000-point tables), E/N 0.1-1000 Td, "
            f"|B| 0-2 T at random angles, I = {args.collisions} real collisions, FP32 flights, FP64 tallies, "
            "windowed trial frequency")


def sweep_name(args):
    return (f"Argon-like E/N sweep: {args.points} log points 1-1000 Td x {max(1, args.electrons // args.scale)} "
            f"electrons x {args.collisions} real collisions, FP32 flights, FP64 tallies, windowed trial "
            "frequency, B = 0" + (f" (point {args.only_point} only)" if args.only_point >= 0 else ""))


def tuned(ctx, mixes, cfgs, args, shared=True, gas_lists=None, headline=False):
    """The autotuner's choice for this batch, or its default options with
    --no-tune (for the headline launch, --block-threads / --smem-budget
    override them).  With several
    ranks and shared=True, rank 0 tunes and every rank takes its choice (the
    legs that follow must agree across ranks).  With gas_lists the tuner may
    choose a table budget; the batch then runs on mixtures compiled for it."""
    from paper_1901_08140_gb300 import autotune
    if args.no_tune:
        choice = dict(autotune.DEFAULT, cached=None)
        if headline and args.block_threads:
            choice["block_threads"] = args.block_threads
        if headline and args.smem_budget and gas_lists is not None:
            choice["smem_budget"] = args.smem_budget
        return choice
    import torch.distributed as dist
    multi = shared and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1
    choice = (autotune.tune(ctx, mixes, cfgs, gas_lists=gas_lists)
              if not multi or dist.get_rank() == 0 else None)
    if multi:
        box = [choice]
        dist.broadcast_object_list(box, src=0)
        choice = box[0]
    return choice


def workload_config(args):
    """The `config` both arms print: the workload, its sizes, the L2 rule."""
    if args.workload == "sweep":
        specs = sweep_specs(args)
        name = sweep_name(args)
    else:
        specs = batched_specs(args)
        name = batched_name(args, specs)
    return specs, {"workload": name, "swarms": len(specs), "electrons": sum(s.n_electrons for s in specs),
                   "real_collisions": args.collisions, "l2": L2_NOTE}


# --------------------------------------------------------------------------
# timing helpers
# --------------------------------------------------------------------------
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


def roofline_of(kind, counts, kern_ms, sm_count, sm_mhz, traffic, kernel):
    """Algorithmic thread operations over the step kernel's time against the
    SMs' issue rate (SMs x 4 schedulers x 32 lanes x SM clock)."""
    ops = ALG_OPS[kind]
    work = (ops["step"] * counts["steps"] + ops["window"] * counts["windows"] + ops["real"] * counts["reals"])
    peak = sm_count * LANES_PER_SM_CLOCK * sm_mhz * 1e6
    achieved = work / (kern_ms / 1e3)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
            "ops_per_unit": ops, "units": counts,
            "note": f"algorithmic thread-ops ({ops['step']}/step + {ops['window']}/window + {ops['real']}/real) "
                    f"over {sm_count} SMs x 128 lanes x median SM clock {sm_mhz:.0f} MHz"}


def counts_of(tallies):
    """Trial steps (real + null + fail + window restarts), new windows (window
    restarts + real collisions + fails) and real collisions."""
    reals = sum(t["n_real"] for t in tallies)
    nulls = sum(t["n_null"] for t in tallies)
    fails = sum(t["n_fail"] for t in tallies)
    wins = sum(t["n_window"] for t in tallies)
    return {"steps": reals + nulls + fails + wins, "windows": wins + reals + fails, "reals": reals,
            "trials": reals + nulls + fails}


# --------------------------------------------------------------------------
# legs of the GPU arm
# --------------------------------------------------------------------------
def batched_run(ctx, stream, flush, world, dev, specs, rank, args, clocks_gpu):
    """The headline: every swarm in one persistent launch replayed from a CUDA
    graph with the autotuner's launch options (and mixtures compiled for its
    table budget); the same swarms one launch each at the same window length
    and the library's default launch shape; the autotuned window length's
    own gain."""
    from paper_1901_08140_gb300 import autotune, bz
    mixes = [bz.Mixture(ctx, s.gases) for s in specs]
    id_off = rank << 32  # weak scaling: every rank runs every swarm on its own ids
    cfgs = [bz.config_from_spec(s, trial_mode=bz.BZ_TRIAL_WINDOW, id_offset=id_off) for s in specs]
    gas_lists = [s.gases for s in specs]
    choice = tuned(ctx, mixes, cfgs, args, gas_lists=gas_lists, headline=True)
    tuned_cfgs = autotune.apply(cfgs, choice)
    bmixes = autotune.mixtures_for(ctx, gas_lists, choice) if choice.get("smem_budget") else mixes
    batch = autotune.make_batch(ctx, bmixes, tuned_cfgs, choice)
    for _ in range(args.warmup):
        batch.launch(stream)
        batch.tallies(check=False)
    clocks = clocks_gpu()
    total_ms = kern_ms = 0.0
    tallies = []
    for _ in range(args.steps):
        ms, _ = _timed(stream, flush, 1, lambda: batch.launch(stream), world, dev)
        total_ms += ms
        ts = batch.tallies()
        tallies += ts
        kern_ms += batch.timing()[0]
    clk = clocks.stop()
    merged = merged_over_ranks(batch, mixes, cfgs, world) if world > 1 else None
    batch.close()
    out = {"ms": total_ms, "kern_ms": kern_ms, "tallies": tallies, "clocks": clk, "choice": choice,
           "merged": merged,
           "mixes": mixes, "cfgs": cfgs, "tuned": tuned_cfgs}
    if "plain" in args.legs:
        def plain_step():
            return [bz.run_swarm(ctx, m, c, stream) for m, c in zip(mixes, tuned_cfgs)]
        for sw in plain_step():
            sw.tallies(check=False)
            sw.close()
        steps = max(1, min(args.steps, 3))
        pms, outs = _timed(stream, flush, steps, plain_step, world, dev)
        preals = 0
        for sws in outs:
            for sw in sws:
                preals += sw.tallies()["n_real"]
                sw.close()
        out["plain"] = {"ms": pms, "steps": steps, "reals": preals}
        # the autotuned window length against the default one, batched both
        if any(abs(c.window_c - 2.0) > 1e-9 for c in tuned_cfgs):
            b2 = autotune.make_batch(ctx, bmixes, cfgs, dict(choice, window_c=2.0))
            b2.launch(stream)
            b2.tallies(check=False)
            dms, _ = _timed(stream, flush, 1, lambda: b2.launch(stream), world, dev)
            dreals = sum(t["n_real"] for t in b2.tallies())
            b2.close()
            out["default_window"] = {"ms": dms, "reals": dreals}
    if bmixes is not mixes:
        for m in bmixes:
            m.close()
    return out


def merged_over_ranks(batch, mixes, cfgs, world):
    """Every swarm's tallies merged over the ranks (each ran its own ids of
    every swarm): the FP64 group sums summed in two all-reduces, so each rank
    holds one set of tallies per swarm over all ranks' electrons."""
    from paper_1901_08140_gb300 import sharding
    out = []
    for i, (m, c) in enumerate(zip(mixes, cfgs)):
        t = sharding.merge_tallies(batch.group_sums1(i), lambda d, i=i: batch.group_sums2(i, d), c.e_over_n_Td,
                                   m.info["n_total"], m.info["nu_trial"])
        out.append(t)
    return {"swarms": len(out), "ranks": world, "electrons": int(sum(t["n_particles"] for t in out)),
            "W_first_swarms": [t["W"] for t in out[:4]], "W_se_first_swarms": [t["W_se"] for t in out[:4]],
            "D_L_first_swarms": [t["D_L"] for t in out[:4]], "D_T_first_swarms": [t["D_T"] for t in out[:4]]}


def e2e_run(ctx, stream, specs, rank, choice, steps):
    """The same metric end to end through the C ABI: per step the mixtures'
    host tables are compiled and copied to the device (16 host threads), the
    swarm configurations copied, the launch run and every swarm's tallies
    read back to the host.  Two steps are in flight: the next step's
    mixtures are compiled and uploaded and its batch set up while the
    current step's launch runs (the first step's set-up is timed alone)."""
    import concurrent.futures as cf
    import torch
    from paper_1901_08140_gb300 import autotune, bz
    id_off = rank << 32
    cfgs = autotune.apply([bz.config_from_spec(s, trial_mode=bz.BZ_TRIAL_WINDOW, id_offset=id_off) for s in specs],
                          choice)
    reals, h2d, d2h = 0, 0, 0
    torch.cuda.synchronize()
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        def prepare():
            mixes = list(ex.map(lambda s: bz.Mixture(ctx, s.gases, smem_budget=int(choice.get("smem_budget", 0))),
                                specs))
            return mixes, autotune.make_batch(ctx, mixes, cfgs, choice)
        nxt = prepare()
        for k in range(steps):
            mixes, b = nxt
            b.launch(stream)
            if k + 1 < steps:
                nxt = prepare()
            ts = b.tallies()
            reals += sum(t["n_real"] for t in ts)
            h2d += sum(m.info["table_bytes"] for m in mixes) + len(cfgs) * (C.sizeof(bz.bz_swarm_config) + 4096)
            d2h += len(cfgs) * C.sizeof(bz.bz_tallies)
            b.close()
            for m in mixes:
                m.close()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # whole job: every rank's real collisions over the slowest rank's time,
    # every rank's bytes
    from paper_1901_08140_gb300 import sharding
    t_max, reals = sharding.reduce_step(dt * 1e3, reals)
    _, h2d = sharding.reduce_step(0.0, h2d)
    _, d2h = sharding.reduce_step(0.0, d2h)
    dt = t_max / 1e3
    return {"value": reals / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d) // steps,
            "d2h_bytes_per_step": int(d2h) // steps,
            "steps": steps, "includes": "mixture compilation and table upload (from pinned host staging), batch set-up, launch, "
                        "tallies read (into pinned host memory)",
            "pipelined": "the next step's mixtures are compiled and uploaded and its batch set up while the "
                         "current step's launch runs; the first step's set-up is timed alone"}


def sweep_run(ctx, stream, flush, world, dev, args, rank):
    """The Argon-like sweep: batched (graph, autotuned) and plain throughput,
    the roofline of its kernel class, the tallies for the oracle check."""
    from paper_1901_08140_gb300 import autotune, bz
    specs = sweep_specs(args)
    mix = bz.Mixture(ctx, specs[0].gases)
    cfgs = [bz.config_from_spec(s, trial_mode=bz.BZ_TRIAL_WINDOW, id_offset=rank << 32) for s in specs]
    choice = tuned(ctx, [mix] * len(cfgs), cfgs, args, shared=False)  # rank 0 alone
    tuned_cfgs = autotune.apply(cfgs, choice)
    batch = autotune.make_batch(ctx, [mix] * len(cfgs), tuned_cfgs, choice)
    for _ in range(2):
        batch.launch(stream)
        batch.tallies()
    steps = max(1, min(args.steps, 5))
    ms = kern = 0.0
    tallies = []
    for _ in range(steps):
        m1, _ = _timed(stream, flush, 1, lambda: batch.launch(stream), world, dev)
        ms += m1
        tallies = batch.tallies()
        kern += batch.timing()[0]
    batch.close()
    pms, outs = _timed(stream, flush, 2, lambda: [bz.run_swarm(ctx, mix, c, stream) for c in tuned_cfgs], world, dev)
    preals = 0
    for sws in outs:
        for sw in sws:
            preals += sw.tallies()["n_real"]
            sw.close()
    reals = sum(t["n_real"] for t in tallies) * steps
    return {"workload": sweep_name(args), "value": reals / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "plain": {"value": preals / (pms / 1e3), "ms_per_step": pms / 2},
            "batched_over_plain": (reals / ms) / (preals / pms),
            "autotuned": {k: choice.get(k) for k in ("window_c", "tiles_per_block", "blocks_per_sm", "channels_in_l2", "block_threads", "smem_budget", "rate_per_ms", "default_rate_per_ms", "cached")},
            "_tallies": tallies, "_kern_ms": kern / steps, "_specs": specs}


def sweep_vs_oracle(sweep_tallies, specs, n_oracle):
    """The sweep's swarm statistics against the FP64 oracle's (the paper's
    constant trial frequency over an energy range it never leaves, so no
    fail biases it) on n_oracle electrons per point with ids after the GPU's:
    relative difference, combined standard error, z-score."""
    from oracle import oracle as O
    from oracle import tallies as OT
    rows = []
    t0 = time.perf_counter()
    for s, g in zip(specs, sweep_tallies):
        m = O.Mixture(s.gases, eps_cap=300.0 if s.e_over_n_Td >= 300.0 else 0.0)
        p = O.run_swarm(m, e_over_n_Td=s.e_over_n_Td, real_collisions=s.real_collisions, n=n_oracle, seed=s.seed,
                        id0=s.n_electrons, threads=O.cpu_count())
        o = OT.swarm_tallies(p, s.e_over_n_Td, m.n_total)
        row = {"E/N_Td": s.e_over_n_Td, "oracle_fails": int(p["n_fail"].sum())}
        for k in ("W", "eps", "D_L", "D_T"):
            se = math.hypot(g[k + "_se"], o[k + "_se"])
            row[k] = {"rel": (g[k] - o[k]) / abs(o[k]), "rel_se": se / abs(o[k]), "z": (g[k] - o[k]) / se}
        rows.append(row)
    summ = {}
    for k in ("W", "eps", "D_L", "D_T"):
        zs = [r[k]["z"] for r in rows]
        resolved = [r for r in rows if 3 * r[k]["rel_se"] <= 0.005]
        summ[k] = {"max_abs_rel": max(abs(r[k]["rel"]) for r in rows), "max_abs_z": max(abs(z) for z in zs),
                   "chi2_over_points": sum(z * z for z in zs), "points_resolving_0.5pct": len(resolved),
                   "resolved_within_0.5pct": sum(1 for r in resolved if abs(r[k]["rel"]) <= 0.005)}
    return {"oracle_electrons_per_point": n_oracle, "gpu_electrons_per_point": specs[0].n_electrons,
            "points": len(rows), "seconds": time.perf_counter() - t0, "summary": summ,
            "max_abs_rel_W": summ["W"]["max_abs_rel"], "per_point": rows}


def batched_vs_oracle(tallies, specs, n_oracle=32000, count=4):
    """Swarms of the timed batched workload (3-4 gases, 30-300 Td, |B| >= 0.3 T,
    at least 1e5 electrons: the first `count` of them) against the FP64
    oracle on n_oracle electrons each, ids after the GPU's: relative
    difference, combined standard error, z-score."""
    from oracle import oracle as O
    from oracle import tallies as OT
    picked = [i for i, s in enumerate(specs) if 30.0 <= s.e_over_n_Td <= 300.0 and len(s.gases) >= 3
              and s.b_T >= 0.3 and s.n_electrons >= 100_000][:count]
    rows = []
    t0 = time.perf_counter()
    for i in picked:
        s, g = specs[i], tallies[i]
        m = O.Mixture(s.gases)
        p = O.run_swarm(m, e_over_n_Td=s.e_over_n_Td, b_T=s.b_T, b_angle_rad=s.b_angle_rad,
                        real_collisions=s.real_collisions, n=n_oracle, seed=s.seed, id0=s.n_electrons,
                        threads=O.cpu_count())
        o = OT.swarm_tallies(p, s.e_over_n_Td, m.n_total)
        row = {"swarm": i, "E/N_Td": s.e_over_n_Td, "B_T": s.b_T, "gases": len(s.gases), "gpu_electrons": s.n_electrons,
               "oracle_fails": int(p["n_fail"].sum())}
        for k in ("W", "eps", "D_L", "D_T"):
            se = math.hypot(g[k + "_se"], o[k + "_se"])
            row[k] = {"rel": (g[k] - o[k]) / abs(o[k]), "rel_se": se / abs(o[k]), "z": (g[k] - o[k]) / se}
        rows.append(row)
    return {"oracle_electrons_per_swarm": n_oracle, "seconds": time.perf_counter() - t0,
            "max_abs_z": max(abs(r[k]["z"]) for r in rows for k in ("W", "eps", "D_L", "D_T")),
            "max_abs_rel_W": max(abs(r["W"]["rel"]) for r in rows), "per_swarm": rows}


def w_qualifier(batched, sweep):
    """The metric's drift-velocity qualifier: the largest |dW|/W against the
    oracle among the comparisons whose samples resolve 0.5 % (three combined
    standard errors below it), beside the figures over every comparison."""
    rows = []
    if batched:
        rows += [("batched swarm %d" % r["swarm"], r["W"]) for r in batched["per_swarm"]]
    if sweep:
        rows += [("sweep %.4g Td" % r["E/N_Td"], r["W"]) for r in sweep["per_point"]]
    if not rows:
        return {}
    res = [(n, w) for n, w in rows if 3 * w["rel_se"] <= 0.005]
    worst = max(res, key=lambda nw: abs(nw[1]["rel"])) if res else None
    return {"max_rel_err_W_vs_oracle": abs(worst[1]["rel"]) if worst else None,
            "w_vs_oracle": {"resolving_0.5pct": len(res), "comparisons": len(rows),
                            "worst_resolved": {"case": worst[0], **worst[1]} if worst else None,
                            "within_0.5pct": sum(1 for _, w in res if abs(w["rel"]) <= 0.005),
                            "max_abs_z_all": max(abs(w["z"]) for _, w in rows),
                            "max_abs_rel_all": max(abs(w["rel"]) for _, w in rows),
                            "note": "relative difference of W from the FP64 oracle (independent ids); the maximum is "
                                    "taken where 3 combined standard errors are below 0.5 %; max_abs_z_all and "
                                    "max_abs_rel_all are over every comparison"}}


def configs_run(ctx, stream):
    """Configurations 1 and 3 on their own: the Maxwell-model gas in FP64
    against its closed forms, and Ar/CO2 90/10 with B = 1 T perpendicular to E."""
    from paper_1901_08140_gb300 import bz
    from paper_1901_08140_gb300 import workloads as W
    QE, ME = 1.602176634e-19, 9.1093837015e-31
    out = {}
    spec = W.maxwell_swarm(n_electrons=10_000, real_collisions=1000)
    mix = bz.Mixture(ctx, spec.gases)
    cfg = bz.config_from_spec(spec)
    best = None
    for _ in range(4):
        sw = bz.run_swarm(ctx, mix, cfg, stream)
        t = sw.tallies()
        ms = sw.timing()[0]
        sw.close()
        best = ms if best is None else min(best, ms)
    g = spec.gases[0]
    vd = QE * spec.e_over_n_Td * 1e-21 * g.number_density_m3 / (ME * 1e12)
    out["maxwell_fp64"] = {"workload": "Maxwell-model gas, E/N = 10 Td, 1e4 electrons x 1000 real collisions, FP64",
                           "value": t["n_real"] / (best / 1e3), "unit": UNIT, "kernel_ms": best,
                           "W_over_vd": t["W"] / vd, "W_se_over_vd": t["W_se"] / vd, "W_flux_over_vd": t["W_flux"] / vd,
                           "eps": t["eps"], "eps_closed_form": 5.2580, "eps_se": t["eps_se"]}
    spec = W.ar_co2_swarm(n_electrons=1_000_000, real_collisions=1000)
    mix = bz.Mixture(ctx, spec.gases)
    cfg = bz.config_from_spec(spec, trial_mode=bz.BZ_TRIAL_WINDOW)
    best = None
    for _ in range(3):
        sw = bz.run_swarm(ctx, mix, cfg, stream)
        t = sw.tallies()
        ms = sw.timing()[0]
        sw.close()
        best = ms if best is None else min(best, ms)
    out["arco2_B1T"] = {"workload": "Ar/CO2 90/10, E/N = 100 Td, B = 1 T perpendicular to E, 1e6 electrons x 1000 "
                                    "real collisions, FP32 flights, windowed trial frequency",
                        "value": t["n_real"] / (best / 1e3), "unit": UNIT, "kernel_ms": best,
                        "W": t["W"], "W_se": t["W_se"], "Wx": t["Wx"], "Wy": t["Wy"],
                        "lorentz_angle_rad": t["lorentz_angle"], "D_L": t["D_L"], "D_L_se": t["D_L_se"],
                        "D_T": t["D_T"], "D_T_se": t["D_T_se"], "efficiency": t["efficiency"]}
    return out


def precision_run(ctx, n):
    """FP32 flights against FP64 throughout on the same swarms (same seeds and
    ids): the Argon-like sweep's 32 points and Ar/CO2 with B = 1 T.  Per
    quantity the largest relative difference and z-score (difference over the
    combined standard error; the two runs draw the same numbers, so they are
    not independent and the z-scores overstate the agreement's spread)."""
    from paper_1901_08140_gb300 import bz
    from paper_1901_08140_gb300 import workloads as W
    out = {}
    for name, specs in (("argon_sweep", W.argon_sweep(n_electrons=n, real_collisions=1000, points=32)),
                        ("arco2_B1T", [W.ar_co2_swarm(n_electrons=n, real_collisions=1000)])):
        mix = bz.Mixture(ctx, specs[0].gases)
        res = {}
        for prec in (32, 64):
            cfgs = [bz.config_from_spec(s, precision=prec, trial_mode=bz.BZ_TRIAL_WINDOW) for s in specs]
            b = bz.Batch(ctx, [mix] * len(cfgs), cfgs, use_graph=False)
            b.launch()
            res[prec] = b.tallies()
            res["ms%d" % prec] = b.timing()[0]
            b.close()
        q = {}
        for k in ("W", "eps", "eps_after", "alpha", "D_L", "D_T"):
            rel, z = [], []
            for a, b64 in zip(res[32], res[64]):
                if b64[k] == 0:
                    continue
                rel.append(abs(a[k] - b64[k]) / abs(b64[k]))
                se = math.hypot(a.get(k + "_se", 0.0) or 0.0, b64.get(k + "_se", 0.0) or 0.0)
                if se > 0:
                    z.append(abs(a[k] - b64[k]) / se)
            q[k] = {"max_rel": max(rel) if rel else None, "median_rel": statistics.median(rel) if rel else None,
                    "max_z": max(z) if z else None}
        out[name] = {"electrons_per_swarm": n, "swarms": len(specs), "fp32_ms": res["ms32"], "fp64_ms": res["ms64"],
                     "quantities": q}
    return out


def strategy_runs(ctx, mix, specs, electrons):
    """The Argon-like sweep at `electrons` per point under each trial frequency
    (Sec. 6): real collisions/s of the step kernel, efficiency (Eq. 28),
    fails, electrons stopped by an error, and the largest deviation of W
    from the exact windowed run in combined standard errors."""
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


def avalanche_runs(ctx, stream, caps):
    """Avalanches alone (the serving workload's avalanche request): one seed
    electron at 300 Td in Ar/CO2 93/7, spawn mode, 1 ns, windowed trial
    frequency, growth capped at each population in `caps`; latency on the
    host clock from the launch to the tallies, and the step kernel's time."""
    from paper_1901_08140_gb300 import bz
    from paper_1901_08140_gb300 import workloads as W
    mix = bz.Mixture(ctx, W.ar_co2_avalanche_mixture())

    def cfg(cap, k):
        return bz.make_config(n_electrons=1, real_collisions=10 ** 9, e_over_n_Td=300.0, seed=W.swarm_seed(5000 + k),
                              t_end_s=1e-9, spawn=True, pop_cap=int(cap), trial_mode=bz.BZ_TRIAL_WINDOW)
    warm = bz.run_swarm(ctx, mix, cfg(1000, 0), stream)
    warm.tallies()
    warm.close()
    out = []
    for k, cap in enumerate(caps):
        t0 = time.perf_counter()
        sw = bz.run_swarm(ctx, mix, cfg(cap, k + 1), stream)
        t = sw.tallies()
        lat = time.perf_counter() - t0
        kms = sw.timing()[0]
        sw.close()
        out.append({"pop_cap": int(cap), "latency_ms": lat * 1e3, "kernel_ms": kms,
                    "final_population": int(t["n_particles"]), "real_collisions": int(t["n_real"]),
                    "real_collisions_per_s": t["n_real"] / (kms / 1e3) if kms > 0 else None,
                    "capped_ionizations": int(t.get("n_capped", 0))})
    return out


def serving_runs(ctx, rates, seconds, collisions=100, pool=64, streams=3, avalanche_frac=0.05,
                 avalanche_cap=100_000, max_group=512):
    """Continuous-batching request loop under Poisson arrivals: swarm sizes,
    mixtures and fields of the batched workload (a pool of compiled
    mixtures), I real collisions per request, windowed trial frequency; a
    fraction are avalanche requests (Ar/CO2 93/7, 300 Td, spawn mode, one
    seed electron, 1 ns, population cap avalanche_cap)."""
    import numpy as np
    from paper_1901_08140_gb300 import bz, serving
    from paper_1901_08140_gb300 import workloads as W
    specs = W.batched_swarms(count=pool, real_collisions=collisions)
    mixes = [bz.Mixture(ctx, s.gases) for s in specs]
    ava_mix = bz.Mixture(ctx, W.ar_co2_avalanche_mixture())
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
        srv = serving.Server(ctx, memory_budget=60e9, n_slots=streams, max_group=max_group)
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
        summ.update({"rate_req_s": rate, "slots": streams, "max_group": max_group,
                     "offered_real_collisions_per_s": offered,
                     "served_fraction": summ["real_collisions_per_s"] / offered if offered else None,
                     "max_concurrent": srv.stats()["max_running"], "launch_groups": srv.stats()["launches"]})
        srv.close()
        out.append(summ)
    return out


def cpu_baseline(args, specs, budget_s):
    """The FP64 oracle, as it stands, on this host's cores: a bounded sample of
    the same swarms -- rounds over the swarms, a block of electrons each with
    ids after the GPU's, until the time bound."""
    from oracle import oracle as O
    cores = O.cpu_count()
    block = 4 * cores
    reals = trials = units = 0
    t0 = time.perf_counter()
    k = 0
    cache = {}
    while time.perf_counter() - t0 < budget_s or units < 2:
        s = specs[k % len(specs)]
        key = id(s.gases)
        if key not in cache:
            cache = {key: O.Mixture(s.gases)}
        p = O.run_swarm(cache[key], e_over_n_Td=s.e_over_n_Td, b_T=s.b_T, b_angle_rad=s.b_angle_rad,
                        real_collisions=s.real_collisions, n=block, seed=s.seed,
                        id0=(1 << 40) + (k // len(specs)) * block, threads=cores)
        reals += int(p["n_real"].sum())
        trials += int(p["n_real"].sum() + p["n_null"].sum() + p["n_fail"].sum())
        units += 1
        k += 1
    dt = time.perf_counter() - t0
    sample = (f"{units} (swarm, {block}-electron id block) units taken round-robin over the {len(specs)} swarms, "
              f"I={specs[0].real_collisions}, FP64, the paper's constant trial frequency; {reals} real / {trials} "
              f"trial collisions in {dt:.1f} s")
    return {"value": reals / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "trial_collisions_per_s": trials / dt}


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
    from paper_1901_08140_gb300 import bz, sharding
    ctx = bz.Context(local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    specs, config = workload_config(args)
    out = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": config}

    # ---- the headline workload
    if args.workload == "batched":
        r = batched_run(ctx, stream, flush, world, dev, specs, rank, args, lambda: Clocks(local))
        bt = int(r["choice"].get("block_threads", 256))
        kind, kernel = "field", (f"batch_kernel (lean FP32 build with the field's paths, {bt} threads x "
                                 f"{768 // bt} blocks/SM, tables compiled for "
                                 f"{int(r['choice'].get('smem_budget', 0)) or 73728} B per block)")
        prof = "batch_kernel_batched_256"
    else:
        from paper_1901_08140_gb300 import autotune
        mix = bz.Mixture(ctx, specs[0].gases)
        cfgs = [bz.config_from_spec(s, trial_mode=bz.BZ_TRIAL_WINDOW, id_offset=rank << 32) for s in specs]
        choice = tuned(ctx, [mix] * len(cfgs), cfgs, args, headline=True)
        tuned_cfgs = autotune.apply(cfgs, choice)
        b = autotune.make_batch(ctx, [mix] * len(cfgs), tuned_cfgs, choice)
        for _ in range(args.warmup):
            b.launch(stream)
            b.tallies()
        clocks = Clocks(local)
        ms = kms = 0.0
        tl = []
        for _ in range(args.steps):
            m1, _ = _timed(stream, flush, 1, lambda: b.launch(stream), world, dev)
            ms += m1
            tl += b.tallies()
            kms += b.timing()[0]
        b.close()
        r = {"ms": ms, "kern_ms": kms, "tallies": tl, "clocks": clocks.stop(), "choice": choice,
             "mixes": [mix] * len(cfgs), "tuned": tuned_cfgs}
        kind, kernel = "plain", "batch_kernel (lean FP32 build without field paths; 4 blocks/SM where the tables fit)"
        prof = "batch_kernel_traffic_argon_sweep"
    reals = sum(t["n_real"] for t in r["tallies"])
    t_max, tot_reals = sharding.reduce_step(r["ms"], reals)
    value = tot_reals / (t_max / 1e3)
    clk = r["clocks"]
    sm_mhz = clk.get("sm_mhz") or 2070.0
    counts = counts_of(r["tallies"])
    out.update({"value": value, "ms_per_step": t_max / args.steps,
                "roofline": roofline_of(kind, counts, r["kern_ms"], sm_count, sm_mhz,
                                        profiled_traffic(prof, {k: r["choice"].get(k, 0) for k in
                                                                ("block_threads", "smem_budget")}), kernel),
                "shared_memory": shared_memory_roofline("batched" if args.workload == "batched" else "sweep",
                                                        counts["reals"], r["kern_ms"], sm_count, sm_mhz,
                                                        {k: r["choice"].get(k, 0) for k in
                                                         ("block_threads", "smem_budget")}),
                "clocks": clk, "gpu_launches": 5 * args.steps,
                "autotuned": {k: r["choice"].get(k) for k in ("window_c", "tiles_per_block", "blocks_per_sm", "channels_in_l2", "block_threads", "smem_budget", "rate_per_ms", "default_rate_per_ms", "cached")},
                "trial_collisions_per_s": counts["trials"] * world / (t_max / 1e3),
                "efficiency": counts["reals"] / counts["trials"] if counts["trials"] else None,
                "window_restarts_per_real": (counts["windows"] - counts["reals"]) / counts["reals"]})
    if r.get("merged"):
        out["merged_tallies"] = r["merged"]
    if "plain" in r:
        p = r["plain"]
        p_max, p_reals = sharding.reduce_step(p["ms"], p["reals"])
        pv = p_reals / (p_max / 1e3)
        out["plain"] = {"value": pv, "ms_per_step": p_max / p["steps"], "steps": p["steps"],
                        "mode": "one persistent launch per swarm, back to back on one stream, the batched "
                                "launch's window length"}
        out["batched_over_plain"] = value / pv
    if "default_window" in r:
        d = r["default_window"]
        out["window_length_gain"] = {"autotuned_window_c": r["choice"]["window_c"],
                                     "batched_at_default_window_c_2": d["reals"] / (d["ms"] / 1e3),
                                     "gain": value / (d["reals"] / (d["ms"] / 1e3))}
    if "e2e" in args.legs:
        out["e2e"] = e2e_run(ctx, stream, specs, rank, r["choice"], min(max(args.steps, 2), 5))
    # ---- further legs (rank 0)
    if rank == 0 and args.workload == "batched" and "oracle" in args.legs and args.scale == 1:
        out["batched_vs_oracle"] = batched_vs_oracle(r["tallies"][-len(specs):], specs, args.batched_oracle_electrons)
    if rank == 0 and args.workload == "batched" and ("sweep" in args.legs or "oracle" in args.legs):
        sw = sweep_run(ctx, stream, flush, 1, dev, args, rank)  # rank 0 alone: no barrier
        sw_counts = counts_of(sw["_tallies"])
        sw["roofline"] = roofline_of("plain", sw_counts, sw["_kern_ms"], sm_count, sm_mhz,
                                     profiled_traffic("batch_kernel_traffic_argon_sweep",
                                                      {k: sw["autotuned"].get(k) for k in ("block_threads", "smem_budget")}),
                                     "batch_kernel (lean FP32 build without field paths; 4 blocks/SM)")
        sw["shared_memory"] = shared_memory_roofline("sweep", sw_counts["reals"], sw["_kern_ms"], sm_count, sm_mhz,
                                                     {k: sw["autotuned"].get(k) for k in
                                                      ("block_threads", "smem_budget")})
        if "oracle" in args.legs:
            sw["drift_velocity_vs_oracle"] = sweep_vs_oracle(sw["_tallies"], sw["_specs"], args.oracle_electrons)
            out.update(w_qualifier(out.get("batched_vs_oracle"), sw["drift_velocity_vs_oracle"]))
        for k in ("_tallies", "_kern_ms", "_specs"):
            sw.pop(k)
        out["argon_sweep"] = sw
    if rank == 0 and "configs" in args.legs:
        out["configurations"] = configs_run(ctx, stream)
    if rank == 0 and "precision" in args.legs:
        out["precision_fp32_vs_fp64"] = precision_run(ctx, args.precision_electrons)
    if rank == 0 and "strategies" in args.legs:
        from paper_1901_08140_gb300 import workloads as W
        ss = W.argon_sweep(points=32)
        out["trial_strategies"] = strategy_runs(ctx, bz.Mixture(ctx, ss[0].gases), ss,
                                                min(args.strategy_electrons, args.electrons))
    if rank == 0 and "avalanche" in args.legs:
        caps = [float(x) for x in args.avalanche_caps.split(",") if x]
        out["avalanche"] = {"workload": "one seed electron, 300 Td, Ar/CO2 93/7, spawn mode, t_end 1 ns, windowed "
                                        "trial frequency, run alone", "runs": avalanche_runs(ctx, stream, caps)}
    if rank == 0 and "serving" in args.legs:
        rates = [float(x) for x in args.serve_rates.split(",") if x]
        serve = serving_runs(ctx, rates, args.serve_seconds, streams=args.serve_slots,
                             avalanche_frac=args.avalanche_frac, avalanche_cap=args.avalanche_cap,
                             max_group=args.serve_max_group)
        out["serving"] = serve
        # the same loop at the workload's own I = 1000 (ten times the work per request)
        rates_long = [float(x) for x in args.serve_rates_i1000.split(",") if x]
        if rates_long:
            out["serving_I1000"] = serving_runs(ctx, rates_long, args.serve_seconds, collisions=1000,
                                                streams=args.serve_slots, avalanche_frac=args.avalanche_frac,
                                                avalanche_cap=args.avalanche_cap, max_group=args.serve_max_group)
        kept = [x for x in serve if x["served_fraction"] is not None and x["served_fraction"] >= 0.9]
        top = max(kept, key=lambda x: x["rate_req_s"]) if kept else None
        out["p99_swarm_latency_ms"] = top["p99_ms"] if top else None
        out["p99_at_rate_req_s"] = top["rate_req_s"] if top else None
        last = max(serve, key=lambda x: x["rate_req_s"])
        out["p99_at_highest_rate"] = {"rate_req_s": last["rate_req_s"], "p99_ms": last["p99_ms"],
                                      "served_fraction": last["served_fraction"],
                                      "saturated": bool((last["served_fraction"] or 0) < 0.9)}
    if rank != 0:
        return
    if "cpu" in args.legs:
        out["cpu_baseline"] = cpu_baseline(args, specs, args.cpu_seconds)
    print(json.dumps(out, default=_jsonable), flush=True)


def run_reference(args):
    """The oracle on this host's cores over the same workload: every step a
    bounded sample of it (a rotating set of swarms, a block of electrons
    each), the paper's constant trial frequency in FP64."""
    world, rank, local = dist()
    if rank != 0:
        return
    from oracle import oracle as O
    specs, config = workload_config(args)
    cores = O.cpu_count()
    block = 4 * cores
    per_step = min(len(specs), 8)
    mixes = {}

    def step(k):
        r = t = 0
        for j in range(per_step):
            i = (k * per_step + j) % len(specs)
            s = specs[i]
            if i not in mixes:
                mixes[i] = O.Mixture(s.gases)
            p = O.run_swarm(mixes[i], e_over_n_Td=s.e_over_n_Td, b_T=s.b_T, b_angle_rad=s.b_angle_rad,
                            real_collisions=s.real_collisions, n=block, seed=s.seed, id0=(1 << 40) + k * block,
                            threads=cores)
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
    sample = (f"per step: {per_step} of the {len(specs)} swarms (taken in turn) x {block} electrons x "
              f"I={specs[0].real_collisions} (FP64 oracle, the paper's constant trial frequency, {cores} threads)")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": config, "sample": sample,
        "trial_collisions_per_s": trials / dt,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out, default=_jsonable), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
