"""Autotuner of the batched step launch.

Picks, for a batch of swarms, the launch options that maximise real
collisions per second of device time: the trial-frequency window length
(``window_c``, windowed mode only; any value samples the same process),
the tile size, expressed as tiles per resident block so that the choice
carries over between a copy of the batch and the batch itself (it sets how
many electrons each lane runs, one after another, per tile), the resident
blocks per SM, the threads per block (256, or 128 / 384 / 768 at the same
register cap where the batch runs the lean FP32 kernel), the
table-staging policy where every mixture could stage its channel tables
(staged, or all channel choices from the cumulative tables in global
memory), and -- for one block of 768 threads per SM, given the swarms' gas
lists -- the shared-memory budget the mixtures' tables are compiled for
(the default fits three blocks per SM; with one block the tables may keep
their densest bucket index and every bin maximum in shared memory).  It times candidates by coordinate descent on a
reduced copy of the batch -- every swarm keeps its mixture, fields and real
collisions per electron but runs half of its electrons, so an electron's
history looks like the full batch's -- checks the winner against the
defaults on the batch itself, and
caches the result in a JSON file keyed by the GPU name and a signature of
the workload (swarm count, electron count, trial modes, precision), so later
runs of the same class skip the search.
"""
from __future__ import annotations

import ctypes as C
import json
import math
import os
from typing import Dict, List, Optional, Sequence

from . import bz

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")

# window_c 1.5 and 16 tiles per block: the fastest point of a full-size sweep of
# the 256-swarm workload on GB300 (window_c 1.0 / 1.5 / 2.0 / 3.0: 2.94 / 2.90 /
# 2.99 / 3.18 s; 8 / 16 / 32 tiles per block: 2.98 / 2.90 / 2.91 s)
DEFAULT = {"window_c": 1.5, "tiles_per_block": 16, "blocks_per_sm": 0, "channels_in_l2": False, "block_threads": 256,
           "smem_budget": 0}
WINDOW_C = [1.0, 1.5, 2.0, 3.0]
TILES_PER_BLOCK = [4, 8, 16, 32]
BLOCKS = [0, 2]
BLOCK_THREADS = [256, 128, 384, 768]
# table budget per block with one block per SM (0: the library's three-block budget)
ONE_BLOCK_BUDGET = 200 * 1024
SM_COUNT = 152
RESIDENT_BLOCKS = 3   # the FP32 step kernel's blocks of 256 threads per SM when its tables fit


def signature(cfgs: Sequence[bz.bz_swarm_config]) -> str:
    """Workload class: number of swarms, log2 of the total electrons, trial modes."""
    total = sum(int(c.n_electrons) for c in cfgs)
    modes = sorted({int(c.trial_mode) for c in cfgs})
    prec = sorted({int(c.precision) for c in cfgs})
    return f"n{len(cfgs)}-e{int(math.log2(max(total, 1)))}-m{'.'.join(map(str, modes))}-p{'.'.join(map(str, prec))}"


def load_cache(path: str = CACHE) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(cache: Dict[str, dict], path: str = CACHE) -> None:
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _copy_cfg(c: bz.bz_swarm_config, **over) -> bz.bz_swarm_config:
    d = bz.bz_swarm_config()
    C.memmove(C.byref(d), C.byref(c), C.sizeof(bz.bz_swarm_config))
    for k, v in over.items():
        setattr(d, k, v)
    return d


def apply(cfgs: Sequence[bz.bz_swarm_config], choice: dict) -> List[bz.bz_swarm_config]:
    """Configurations with the chosen window length (windowed swarms only)."""
    return [_copy_cfg(c, window_c=float(choice["window_c"])) if c.trial_mode == bz.BZ_TRIAL_WINDOW else c
            for c in cfgs]


def tile_size(cfgs: Sequence[bz.bz_swarm_config], choice: dict, sm_count: int = SM_COUNT) -> int:
    """Electrons per tile for `tiles_per_block` tiles per resident block
    (rounded up to 256, at least 256)."""
    total = sum(int(c.n_electrons) for c in cfgs)
    bps = int(choice.get("blocks_per_sm", 0)) or RESIDENT_BLOCKS * 256 // int(choice.get("block_threads", 256))
    t = math.ceil(total / (sm_count * bps * int(choice.get("tiles_per_block", 16))))
    return max(256, (t + 255) // 256 * 256)


def mixtures_for(ctx, gas_lists: Sequence, choice: dict) -> List["bz.Mixture"]:
    """One mixture per gas list, compiled for the choice's table budget."""
    return [bz.Mixture(ctx, g, smem_budget=int(choice.get("smem_budget", 0))) for g in gas_lists]


def make_batch(ctx, mixtures, cfgs, choice, use_graph: bool = True, sm_count: int = SM_COUNT) -> "bz.Batch":
    """A batch launched with the chosen options (cfgs already carry the
    chosen window length, see apply)."""
    return bz.Batch(ctx, mixtures, cfgs, tile_particles=tile_size(cfgs, choice, sm_count),
                    blocks_per_sm=int(choice.get("blocks_per_sm", 0)), use_graph=use_graph,
                    channels_in_l2=bool(choice.get("channels_in_l2", False)),
                    block_threads=int(choice.get("block_threads", 256)))


def _measure(ctx, mixtures, cfgs, choice, sm_count, repeats=2) -> float:
    """Real collisions per millisecond of step-kernel time (best of `repeats`)."""
    b = make_batch(ctx, mixtures, apply(cfgs, choice), choice, sm_count=sm_count)
    best = 0.0
    for _ in range(repeats):
        b.launch()
        reals = sum(t["n_real"] for t in b.tallies(check=False))
        ms, _ = b.timing()
        best = max(best, reals / max(ms, 1e-6))
    b.close()
    return best


def _try_measure(ctx, mixtures, cfgs, choice, sm_count) -> float:
    """_measure, or 0 for a candidate the library rejects (for example a
    block size whose tables cannot be resident)."""
    try:
        return _measure(ctx, mixtures, cfgs, choice, sm_count)
    except bz.BzError:
        return 0.0


def tune(ctx, mixtures: Sequence, cfgs: Sequence[bz.bz_swarm_config], scale: float = 0.5,
         use_cache: bool = True, cache_path: str = CACHE, gpu_name: Optional[str] = None,
         margin: float = 0.02, gas_lists: Optional[Sequence] = None) -> dict:
    """Best launch options for this batch (cached per GPU and workload class).

    mixtures were compiled with the library's default table budget; with
    gas_lists (the gases of each swarm's mixture) the tuner may also choose
    a larger budget, and the caller then runs the batch on mixtures_for(...).
    A candidate replaces the current best only if it is faster by more than
    `margin` on the reduced copy; at the end the choice and the defaults are
    timed once each on the batch itself and the faster is kept, so the
    tuner never settles on options slower than the defaults."""
    import torch
    if gpu_name is None:
        gpu_name = torch.cuda.get_device_name(ctx.device)
    key = f"{gpu_name}|{signature(cfgs)}"
    cache = load_cache(cache_path) if use_cache else {}
    if key in cache and "smem_budget" in cache[key]:
        hit = dict(cache[key], cached=True)
        if gas_lists is None:
            hit["smem_budget"] = 0  # the caller cannot compile mixtures for another budget
        return hit
    sm_count = torch.cuda.get_device_properties(ctx.device).multi_processor_count
    small = [_copy_cfg(c, n_electrons=max(256, int(c.n_electrons * scale))) for c in cfgs]
    best = dict(DEFAULT)
    best_rate = _measure(ctx, mixtures, small, best, sm_count)
    windowed = any(c.trial_mode == bz.BZ_TRIAL_WINDOW for c in cfgs)
    # the staging policy matters only where every mixture would stage its channel tables
    staged = all(m.info.get("channels_in_smem") for m in mixtures) and all(int(c.precision) == 32 for c in cfgs)
    # other block sizes are built for the lean FP32 kernel only
    lean = (all(int(c.precision) == 32 for c in cfgs)
            and all(int(c.trial_mode) not in (bz.BZ_TRIAL_VARIABLE, bz.BZ_TRIAL_BINNED) for c in cfgs)
            and not any(m.info.get("n_xi_gases") for m in mixtures))
    for name, values in (("window_c", WINDOW_C if windowed else []), ("tiles_per_block", TILES_PER_BLOCK),
                         ("blocks_per_sm", BLOCKS), ("channels_in_l2", [False, True] if staged else []),
                         ("block_threads", BLOCK_THREADS if lean else [])):
        for v in values:
            if v == best[name]:
                continue
            cand = dict(best, **{name: v})
            r = _try_measure(ctx, mixtures, small, cand, sm_count)
            if r > best_rate * (1.0 + margin):
                best, best_rate = cand, r
    big = None
    if gas_lists is not None and lean:
        # one block of 768 threads per SM with tables compiled for it
        big = mixtures_for(ctx, gas_lists, {"smem_budget": ONE_BLOCK_BUDGET})
        cand = dict(best, block_threads=768, blocks_per_sm=0, smem_budget=ONE_BLOCK_BUDGET)
        r = _try_measure(ctx, big, small, cand, sm_count)
        if r > best_rate * (1.0 + margin):
            best, best_rate = cand, r
    best["rate_per_ms_reduced"] = best_rate
    if any(best[k] != DEFAULT[k] for k in DEFAULT):
        full_best = _measure(ctx, big if best["smem_budget"] else mixtures, cfgs, best, sm_count, repeats=1)
        full_default = _measure(ctx, mixtures, cfgs, DEFAULT, sm_count, repeats=1)
        if full_default >= full_best:
            best = dict(DEFAULT, rate_per_ms_reduced=best_rate, rejected=dict(best))
        best["rate_per_ms"] = max(full_best, full_default)
        best["default_rate_per_ms"] = full_default
    for m in big or []:
        m.close()
    cache[key] = best
    if use_cache:
        store_cache(cache, cache_path)
    return dict(best, cached=False)
