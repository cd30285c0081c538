"""Python binding of libbz.so: argument marshalling only.

The functions ``bz_*`` mirror include/bz.h one to one.  The helpers below
them (``Context``, ``Mixture``, ``run_swarm`` ...) only pack numpy / torch
data into the C structs; every step of the transport method runs in the
library's CUDA kernels.  PyTorch provides device memory (its caching
allocator backs the library's allocator callbacks) and streams.

There is no CPU fallback: if libbz.so is missing or no CUDA device is
present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import sys
from typing import Dict, Optional, Sequence

import numpy as np

from . import build as _build

BZ_OK, BZ_EINVAL, BZ_ENOMEM, BZ_EBUDGET, BZ_ETRIAL, BZ_ETIMEOUT, BZ_ECUDA, BZ_ECANCEL, BZ_ENOTREADY = range(9)
BZ_TRIAL_LAZY, BZ_TRIAL_FIXED, BZ_TRIAL_WINDOW, BZ_TRIAL_VARIABLE, BZ_TRIAL_BINNED = 0, 1, 2, 3, 4
DEC_WINDOW, DEC_FAIL, DEC_NULL = -3, -2, -1
ST_DONE, ST_TIME, ST_STEPS, ST_TRIAL, ST_ERROR, ST_ATTACHED = 0, 1, 2, 3, 4, 5
BZ_ERR_STAGE_TIMEOUT, BZ_ERR_TRIAL, BZ_ERR_NONFINITE, BZ_ERR_MAX_TRIALS, BZ_ERR_SPAWN_WAIT = 1, 2, 4, 8, 16


class BzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"bz status {status}: {msg}")
        self.status = status


# --------------------------------------------------------------------------
# C structs (layout of include/bz.h)
# --------------------------------------------------------------------------
class bz_channel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_points", C.c_int32), ("threshold_eV", C.c_double),
                ("energy_eV", C.POINTER(C.c_double)), ("sigma_m2", C.POINTER(C.c_double))]


class bz_gas(C.Structure):
    _fields_ = [("mass_kg", C.c_double), ("number_density_m3", C.c_double), ("angular", C.c_int32),
                ("n_channels", C.c_int32), ("channels", C.POINTER(bz_channel)), ("el_n_points", C.c_int32),
                ("reserved", C.c_int32), ("el_energy_eV", C.POINTER(C.c_double)),
                ("sigma_el_m2", C.POINTER(C.c_double))]


class bz_mixture_opts(C.Structure):
    _fields_ = [("eps_cap_eV", C.c_double), ("majorant_guard", C.c_double), ("channels_in_smem", C.c_int32),
                ("smem_budget", C.c_int32)]


class bz_mixture_info(C.Structure):
    _fields_ = [("nu_max", C.c_double), ("nu_trial", C.c_double), ("eps_at_max", C.c_double),
                ("eps_cap", C.c_double), ("n_total", C.c_double), ("n_gases", C.c_int32),
                ("n_channels", C.c_int32), ("n_records", C.c_int32), ("n_buckets", C.c_int32),
                ("smem_bytes", C.c_int32), ("channels_in_smem", C.c_int32), ("first_tail_record", C.c_int32),
                ("table_bytes", C.c_int32), ("n_xi_gases", C.c_int32), ("reserved", C.c_int32)]


class bz_swarm_config(C.Structure):
    _fields_ = [("e_over_n_Td", C.c_double), ("b_T", C.c_double), ("b_angle_rad", C.c_double),
                ("n_electrons", C.c_uint64), ("real_collisions", C.c_uint32), ("precision", C.c_int32),
                ("trial_mode", C.c_int32), ("attach_keep_state", C.c_int32), ("nu_trial", C.c_double),
                ("eps0_mean_eV", C.c_double), ("t_end_s", C.c_double), ("max_trials", C.c_uint64),
                ("seed", C.c_uint64), ("id_offset", C.c_uint64), ("block_threads", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("window_c", C.c_double), ("spawn", C.c_int32),
                ("reserved0", C.c_int32), ("pop_cap", C.c_uint64), ("zeta", C.c_double),
                ("grace", C.c_uint32), ("bins_per_decade", C.c_int32), ("gas_temperature_K", C.c_double),
                ("spawn_wait_s", C.c_double), ("hold_pending", C.c_uint32), ("hold_stage", C.c_uint32),
                ("stage_wait_s", C.c_double)]


_TALLY_DOUBLES = ["W", "W_se", "Wx", "Wy", "W_flux", "lorentz_angle", "mu", "mu_N", "mu_0", "eps", "eps_se",
                  "eps_after", "eps_after_se", "alpha", "alpha_se", "eta", "eta_se", "alpha_flux", "eta_flux",
                  "D", "D_se", "D_L", "D_L_se", "D_T", "D_T_se", "D_L_flux", "D_T_flux", "sig", "sig_se",
                  "sig_L", "sig_L_se", "sig_T", "sig_T_se", "efficiency", "E_V_m", "n_total", "nu_trial",
                  "t_mean"]
_TALLY_COUNTS = ["n_particles", "n_real", "n_null", "n_fail", "n_ion", "n_att", "n_incomplete", "n_window",
                 "n_spawned", "n_alive", "n_removed", "n_capped"]


class bz_tallies(C.Structure):
    _fields_ = [(k, C.c_double) for k in _TALLY_DOUBLES] + [(k, C.c_uint64) for k in _TALLY_COUNTS] + \
        [("error_flags", C.c_int32), ("reserved", C.c_int32)]


_PART_D = ["x", "y", "z", "t", "sum_e", "sum_e2"]
_PART_F = ["vx", "vy", "vz", "nu_p"]
_PART_U = ["n_real", "n_null", "n_fail", "n_ion", "n_att", "steps", "status"]


class bz_particles(C.Structure):
    _fields_ = [(k, C.POINTER(C.c_double)) for k in _PART_D] + [(k, C.POINTER(C.c_float)) for k in _PART_F] + \
        [(k, C.POINTER(C.c_uint32)) for k in _PART_U] + [("id", C.POINTER(C.c_uint64)),
                                                        ("t_birth", C.POINTER(C.c_double))]


class bz_particle_arrays(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ["x", "y", "z", "t", "sum_e", "sum_e2", "n_real", "n_null", "n_fail",
                                          "n_ion", "n_att", "status", "steps"]]


BZ_NOALLOC_MAX_PARTICLES = 32768 * 512


class bz_batch_opts(C.Structure):
    _fields_ = [("tile_particles", C.c_int32), ("blocks_per_sm", C.c_int32), ("use_graph", C.c_int32),
                ("channels_in_l2", C.c_int32), ("block_threads", C.c_int32)]


class bz_merge_info(C.Structure):
    _fields_ = [("e_over_n_Td", C.c_double), ("n_total_m3", C.c_double), ("nu_trial", C.c_double),
                ("n_spawned", C.c_uint64), ("n_capped", C.c_uint64), ("error_flags", C.c_int32),
                ("reserved", C.c_int32)]


BZ_GROUPS, BZ_GROUP_Q1, BZ_GROUP_Q2 = 32, 21, 8


class bz_server_opts(C.Structure):
    _fields_ = [("memory_budget_bytes", C.c_double), ("n_slots", C.c_int32), ("max_group", C.c_int32),
                ("simulate", C.c_int32), ("reserved", C.c_int32)]


class bz_request_info(C.Structure):
    _fields_ = [("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("launch", C.c_uint64), ("group_size", C.c_int32), ("status", C.c_int32)]


class bz_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("cancelled", C.c_uint64),
                ("launches", C.c_uint64), ("queued", C.c_int32), ("running", C.c_int32),
                ("max_running", C.c_int32), ("reserved", C.c_int32), ("bytes_in_use", C.c_double),
                ("peak_bytes_in_use", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class bz_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


# --------------------------------------------------------------------------
# Library
# --------------------------------------------------------------------------
_lib = None

# name -> (restype, argtypes): every function declared in include/bz.h
SIGNATURES = {
    "bz_create": (C.c_int, [C.c_int, C.POINTER(bz_allocator), C.POINTER(C.c_void_p)]),
    "bz_destroy": (None, [C.c_void_p]),
    "bz_last_error": (C.c_char_p, []),
    "bz_abi_version": (C.c_int, []),
    "bz_create_gas_mixture": (C.c_int, [C.c_void_p, C.POINTER(bz_gas), C.c_int32, C.POINTER(bz_mixture_opts),
                                        C.POINTER(C.c_void_p)]),
    "bz_destroy_mixture": (None, [C.c_void_p]),
    "bz_mixture_get_info": (C.c_int, [C.c_void_p, C.POINTER(bz_mixture_info)]),
    "bz_mixture_compile_info": (C.c_int, [C.POINTER(bz_gas), C.c_int32, C.POINTER(bz_mixture_opts),
                                          C.POINTER(bz_mixture_info)]),
    "bz_config_defaults": (None, [C.POINTER(bz_swarm_config)]),
    "bz_set_fields": (C.c_int, [C.POINTER(bz_swarm_config), C.c_double, C.c_double, C.c_double]),
    "bz_run_swarm": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(bz_swarm_config), C.c_void_p,
                               C.POINTER(C.c_void_p)]),
    "bz_read_tallies": (C.c_int, [C.c_void_p, C.POINTER(bz_tallies)]),
    "bz_query_tallies": (C.c_int, [C.c_void_p, C.POINTER(bz_tallies)]),
    "bz_read_particles": (C.c_int, [C.c_void_p, C.POINTER(bz_particles)]),
    "bz_destroy_swarm": (None, [C.c_void_p]),
    "bz_swarm_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "bz_swarm_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "bz_create_batch": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p), C.POINTER(bz_swarm_config),
                                  C.POINTER(bz_batch_opts), C.POINTER(C.c_void_p)]),
    "bz_launch_batch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bz_batch_query": (C.c_int, [C.c_void_p]),
    "bz_batch_read_tallies": (C.c_int, [C.c_void_p, C.POINTER(bz_tallies)]),
    "bz_batch_read_particles": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(bz_particles)]),
    "bz_batch_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "bz_destroy_batch": (None, [C.c_void_p]),
    "bz_reduce_tallies_noalloc": (C.c_int, [C.POINTER(bz_particle_arrays), C.c_uint64, C.c_uint64, C.c_double,
                                            C.c_double, C.c_double, C.c_void_p, C.c_void_p]),
    "bz_swarm_group_sums1": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bz_swarm_group_sums2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "bz_batch_group_sums1": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "bz_batch_group_sums2": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "bz_drift_from_group_sums": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bz_finalize_group_sums": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(bz_merge_info), C.POINTER(bz_tallies)]),
    "bz_server_create": (C.c_int, [C.c_void_p, C.POINTER(bz_server_opts), C.POINTER(C.c_void_p)]),
    "bz_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(bz_swarm_config), C.POINTER(C.c_uint64)]),
    "bz_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(bz_tallies), C.POINTER(bz_request_info)]),
    "bz_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "bz_server_pause": (C.c_int, [C.c_void_p, C.c_int32]),
    "bz_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(bz_server_stats)]),
    "bz_server_destroy": (None, [C.c_void_p]),
    "bz_step_replay": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(bz_swarm_config), C.c_int64, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bz_philox": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libbz.so; raises if it has not been built (no CPU fallback)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise BzError(BZ_ECUDA, f"{path} is missing: build it with paper_1901_08140_gb300.build.build()")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != BZ_OK:
        raise BzError(status, lib().bz_last_error().decode())


# Same-name pass-throughs of the C ABI.
def bz_create(device, alloc, out): return lib().bz_create(device, alloc, out)
def bz_destroy(ctx): return lib().bz_destroy(ctx)
def bz_last_error(): return lib().bz_last_error().decode()
def bz_abi_version(): return lib().bz_abi_version()
def bz_create_gas_mixture(ctx, gases, n, opts, out): return lib().bz_create_gas_mixture(ctx, gases, n, opts, out)
def bz_destroy_mixture(m): return lib().bz_destroy_mixture(m)
def bz_mixture_get_info(m, out): return lib().bz_mixture_get_info(m, out)
def bz_mixture_compile_info(gases, n, opts, out): return lib().bz_mixture_compile_info(gases, n, opts, out)
def bz_config_defaults(cfg): return lib().bz_config_defaults(cfg)
def bz_set_fields(cfg, eon, b, ang): return lib().bz_set_fields(cfg, eon, b, ang)
def bz_run_swarm(ctx, m, cfg, stream, out): return lib().bz_run_swarm(ctx, m, cfg, stream, out)
def bz_read_tallies(sw, out): return lib().bz_read_tallies(sw, out)
def bz_query_tallies(sw, out): return lib().bz_query_tallies(sw, out)
def bz_read_particles(sw, out): return lib().bz_read_particles(sw, out)
def bz_destroy_swarm(sw): return lib().bz_destroy_swarm(sw)
def bz_swarm_timing(sw, a, b): return lib().bz_swarm_timing(sw, a, b)
def bz_swarm_size(sw, n): return lib().bz_swarm_size(sw, n)
def bz_create_batch(*a): return lib().bz_create_batch(*a)
def bz_launch_batch(b, stream): return lib().bz_launch_batch(b, stream)
def bz_batch_query(b): return lib().bz_batch_query(b)
def bz_batch_read_tallies(b, out): return lib().bz_batch_read_tallies(b, out)
def bz_batch_read_particles(b, i, out): return lib().bz_batch_read_particles(b, i, out)
def bz_batch_timing(b, a, c): return lib().bz_batch_timing(b, a, c)
def bz_destroy_batch(b): return lib().bz_destroy_batch(b)
def bz_reduce_tallies_noalloc(*a): return lib().bz_reduce_tallies_noalloc(*a)
def bz_swarm_group_sums1(sw, out): return lib().bz_swarm_group_sums1(sw, out)
def bz_swarm_group_sums2(sw, drift, out): return lib().bz_swarm_group_sums2(sw, drift, out)
def bz_batch_group_sums1(b, i, out): return lib().bz_batch_group_sums1(b, i, out)
def bz_batch_group_sums2(b, i, drift, out): return lib().bz_batch_group_sums2(b, i, drift, out)
def bz_drift_from_group_sums(g1, drift): return lib().bz_drift_from_group_sums(g1, drift)
def bz_finalize_group_sums(g1, g2, info, out): return lib().bz_finalize_group_sums(g1, g2, info, out)
def bz_server_create(ctx, opts, out): return lib().bz_server_create(ctx, opts, out)
def bz_submit(srv, mix, cfg, rid): return lib().bz_submit(srv, mix, cfg, rid)
def bz_poll(srv, rid, out, info): return lib().bz_poll(srv, rid, out, info)
def bz_cancel(srv, rid): return lib().bz_cancel(srv, rid)
def bz_server_pause(srv, paused): return lib().bz_server_pause(srv, paused)
def bz_server_get_stats(srv, out): return lib().bz_server_get_stats(srv, out)
def bz_server_destroy(srv): return lib().bz_server_destroy(srv)
def bz_step_replay(*a): return lib().bz_step_replay(*a)
def bz_philox(*a): return lib().bz_philox(*a)


# --------------------------------------------------------------------------
# Helpers
# --------------------------------------------------------------------------
def _torch():
    import torch
    if not torch.cuda.is_available():
        raise BzError(BZ_ECUDA, "no CUDA device: libbz.so has no CPU fallback")
    return torch


def _stream_handle(stream) -> int:
    torch = _torch()
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Context:
    """A bz_ctx on one device whose device memory comes from PyTorch."""

    def __init__(self, device: int = 0, torch_allocator: bool = True):
        torch = _torch()
        self.device = device
        torch.cuda.set_device(device)
        self._alloc = None
        if torch_allocator:
            dev = device

            def _a(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or None)
                except Exception:  # out of memory: the library reports BZ_ENOMEM
                    return None

            def _f(ptr, nbytes, stream, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (ALLOC_FN(_a), FREE_FN(_f))
            self._alloc = bz_allocator(self._cb[0], self._cb[1], None)
        h = C.c_void_p()
        _check(lib().bz_create(device, C.byref(self._alloc) if self._alloc is not None else None, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().bz_destroy(self.h)
            self.h = None

    def __del__(self):
        # at interpreter shutdown the allocator callbacks may already be gone
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def _gas_structs(gases):
    keep = []
    gs = (bz_gas * len(gases))()
    for i, g in enumerate(gases):
        chs = (bz_channel * len(g.channels))()
        for j, ch in enumerate(g.channels):
            e = np.ascontiguousarray(ch.energy_eV, dtype=np.float64)
            s = np.ascontiguousarray(ch.sigma_m2, dtype=np.float64)
            keep += [e, s]
            chs[j] = bz_channel(int(ch.kind), len(e), float(ch.threshold_eV),
                                e.ctypes.data_as(C.POINTER(C.c_double)), s.ctypes.data_as(C.POINTER(C.c_double)))
        keep.append(chs)
        gs[i] = bz_gas(float(g.mass_kg), float(g.number_density_m3), int(g.angular), len(g.channels), chs)
        el = getattr(g, "sigma_el", None)
        if el is not None:
            ee = np.ascontiguousarray(el[0], dtype=np.float64)
            es = np.ascontiguousarray(el[1], dtype=np.float64)
            keep += [ee, es]
            gs[i].el_n_points = len(ee)
            gs[i].el_energy_eV = ee.ctypes.data_as(C.POINTER(C.c_double))
            gs[i].sigma_el_m2 = es.ctypes.data_as(C.POINTER(C.c_double))
    return gs, keep


class Mixture:
    """Compiled gas mixture on the device (bz_create_gas_mixture)."""

    def __init__(self, ctx: Context, gases, eps_cap_eV: float = 0.0, majorant_guard: float = -1.0,
                 channels_in_smem: int = -1, smem_budget: int = 0):
        self.ctx = ctx
        gs, keep = _gas_structs(gases)
        opts = bz_mixture_opts(float(eps_cap_eV), float(majorant_guard), int(channels_in_smem), int(smem_budget))
        h = C.c_void_p()
        _check(lib().bz_create_gas_mixture(ctx.h, gs, len(gases), C.byref(opts), C.byref(h)))
        del keep
        self.h = h
        info = bz_mixture_info()
        _check(lib().bz_mixture_get_info(h, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in bz_mixture_info._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().bz_destroy_mixture(self.h)
            self.h = None

    def __del__(self):
        # at interpreter shutdown the allocator callbacks may already be gone
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def compile_info(gases, eps_cap_eV: float = 0.0, majorant_guard: float = -1.0) -> Dict[str, float]:
    """Host-only mixture compilation (bz_mixture_compile_info): no device needed."""
    gs, keep = _gas_structs(gases)
    opts = bz_mixture_opts(float(eps_cap_eV), float(majorant_guard), -1, 0)
    info = bz_mixture_info()
    _check(lib().bz_mixture_compile_info(gs, len(gases), C.byref(opts), C.byref(info)))
    del keep
    return {k: getattr(info, k) for k, _ in bz_mixture_info._fields_}


def make_config(*, n_electrons: int, real_collisions: int, e_over_n_Td: float, b_T: float = 0.0,
                b_angle_rad: float = 0.0, precision: int = 32, seed: int = 1901081400, eps0_mean_eV: float = 0.1,
                trial_mode: int = BZ_TRIAL_LAZY, nu_trial: float = 0.0, t_end_s: float = 0.0, max_trials: int = 0,
                id_offset: int = 0, attach_keep_state: bool = False, blocks_per_sm: int = 0,
                window_c: float = 0.0, spawn: bool = False, pop_cap: int = 0, zeta: float = 0.25,
                grace: int = 5000, bins_per_decade: int = 8, gas_temperature_K: float = 0.0,
                spawn_wait_s: float = 0.0, hold_pending: int = 0, stage_wait_s: float = 0.0,
                hold_stage: int = 0) -> bz_swarm_config:
    cfg = bz_swarm_config()
    lib().bz_config_defaults(C.byref(cfg))
    _check(lib().bz_set_fields(C.byref(cfg), float(e_over_n_Td), float(b_T), float(b_angle_rad)))
    cfg.n_electrons = int(n_electrons)
    cfg.real_collisions = int(real_collisions)
    cfg.precision = int(precision)
    cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    cfg.eps0_mean_eV = float(eps0_mean_eV)
    cfg.trial_mode = int(trial_mode)
    cfg.nu_trial = float(nu_trial)
    cfg.t_end_s = float(t_end_s)
    cfg.max_trials = int(max_trials)
    cfg.id_offset = int(id_offset)
    cfg.attach_keep_state = int(bool(attach_keep_state))
    cfg.blocks_per_sm = int(blocks_per_sm)
    cfg.window_c = float(window_c)
    cfg.spawn = int(bool(spawn))
    cfg.pop_cap = int(pop_cap)
    cfg.zeta = float(zeta)
    cfg.grace = int(grace)
    cfg.bins_per_decade = int(bins_per_decade)
    cfg.gas_temperature_K = float(gas_temperature_K)
    cfg.spawn_wait_s = float(spawn_wait_s)
    cfg.hold_pending = int(hold_pending)
    cfg.stage_wait_s = float(stage_wait_s)
    cfg.hold_stage = int(hold_stage)
    return cfg


def config_from_spec(spec, **over) -> bz_swarm_config:
    kw = dict(n_electrons=spec.n_electrons, real_collisions=spec.real_collisions, e_over_n_Td=spec.e_over_n_Td,
              b_T=spec.b_T, b_angle_rad=spec.b_angle_rad, precision=spec.precision, seed=spec.seed,
              eps0_mean_eV=spec.eps0_mean_eV)
    kw.update(over)
    return make_config(**kw)


class Swarm:
    """A launched swarm (bz_run_swarm); results are read on demand."""

    def __init__(self, ctx: Context, mix: Mixture, cfg: bz_swarm_config, stream=None):
        self.ctx, self.mix, self.cfg = ctx, mix, cfg
        h = C.c_void_p()
        _check(lib().bz_run_swarm(ctx.h, mix.h, C.byref(cfg), C.c_void_p(_stream_handle(stream)), C.byref(h)))
        self.h = h

    def tallies(self, check: bool = True) -> Dict[str, float]:
        t = bz_tallies()
        st = lib().bz_read_tallies(self.h, C.byref(t))
        if check:
            _check(st)
        out = {k: getattr(t, k) for k in _TALLY_DOUBLES + _TALLY_COUNTS}
        out["error_flags"] = t.error_flags
        out["status"] = st
        return out

    def size(self) -> int:
        n = C.c_uint64()
        _check(lib().bz_swarm_size(self.h, C.byref(n)))
        return int(n.value)

    def particles(self) -> Dict[str, np.ndarray]:
        n = self.size()
        arrs, p = _particle_arrays(n)
        _check(lib().bz_read_particles(self.h, C.byref(p)))
        return arrs

    def group_sums1(self) -> np.ndarray:
        """Pass-1 group sums (32 x 21) of the finished swarm."""
        out = np.zeros((BZ_GROUPS, BZ_GROUP_Q1))
        _check(lib().bz_swarm_group_sums1(self.h, out.ctypes.data))
        return out

    def group_sums2(self, drift) -> np.ndarray:
        """Pass-2 group sums (32 x 8) about the drift vector `drift` (6 values)."""
        d = np.ascontiguousarray(drift, dtype=np.float64)
        out = np.zeros((BZ_GROUPS, BZ_GROUP_Q2))
        _check(lib().bz_swarm_group_sums2(self.h, d.ctypes.data, out.ctypes.data))
        return out

    def timing(self):
        """(step kernel ms, tally kernels ms) from CUDA events on the swarm's stream."""
        a, b = C.c_double(), C.c_double()
        _check(lib().bz_swarm_timing(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "h", None):
            lib().bz_destroy_swarm(self.h)
            self.h = None

    def __del__(self):
        # at interpreter shutdown the allocator callbacks may already be gone
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def _tally_dict(t) -> Dict[str, float]:
    out = {k: getattr(t, k) for k in _TALLY_DOUBLES + _TALLY_COUNTS}
    out["error_flags"] = t.error_flags
    return out


def _particle_arrays(n: int):
    arrs = {k: np.zeros(n, np.float64) for k in _PART_D}
    arrs.update({k: np.zeros(n, np.float32) for k in _PART_F})
    arrs.update({k: np.zeros(n, np.uint32) for k in _PART_U})
    arrs["id"] = np.zeros(n, np.uint64)
    arrs["t_birth"] = np.zeros(n, np.float64)
    p = bz_particles(*[arrs[k].ctypes.data_as(C.POINTER(C.c_double)) for k in _PART_D],
                     *[arrs[k].ctypes.data_as(C.POINTER(C.c_float)) for k in _PART_F],
                     *[arrs[k].ctypes.data_as(C.POINTER(C.c_uint32)) for k in _PART_U],
                     arrs["id"].ctypes.data_as(C.POINTER(C.c_uint64)),
                     arrs["t_birth"].ctypes.data_as(C.POINTER(C.c_double)))
    return arrs, p


class Batch:
    """Many swarms in one persistent launch (bz_create_batch / bz_launch_batch)."""

    def __init__(self, ctx: Context, mixtures: Sequence["Mixture"], cfgs: Sequence[bz_swarm_config],
                 tile_particles: int = 0, blocks_per_sm: int = 0, use_graph: bool = True,
                 channels_in_l2: bool = False, block_threads: int = 0):
        self.ctx, self.mixtures, self.n = ctx, list(mixtures), len(cfgs)
        self.cfgs = (bz_swarm_config * self.n)(*cfgs)
        mh = (C.c_void_p * self.n)(*[m.h.value for m in mixtures])
        opts = bz_batch_opts(int(tile_particles), int(blocks_per_sm), int(bool(use_graph)), int(bool(channels_in_l2)),
                             int(block_threads))
        h = C.c_void_p()
        _check(lib().bz_create_batch(ctx.h, self.n, mh, self.cfgs, C.byref(opts), C.byref(h)))
        self.h = h

    def launch(self, stream=None):
        _check(lib().bz_launch_batch(self.h, C.c_void_p(_stream_handle(stream))))

    def ready(self) -> bool:
        st = lib().bz_batch_query(self.h)
        if st == BZ_ENOTREADY:
            return False
        _check(st)
        return True

    def tallies(self, check: bool = True):
        out = (bz_tallies * self.n)()
        st = lib().bz_batch_read_tallies(self.h, out)
        if check:
            _check(st)
        return [_tally_dict(t) for t in out]

    def particles(self, i: int) -> Dict[str, np.ndarray]:
        n = int(self.cfgs[i].n_electrons)
        arrs, p = _particle_arrays(n)
        _check(lib().bz_batch_read_particles(self.h, int(i), C.byref(p)))
        off = int(self.cfgs[i].id_offset)
        arrs["id"] = np.arange(off, off + n, dtype=np.uint64)
        return arrs

    def timing(self):
        a, b = C.c_double(), C.c_double()
        _check(lib().bz_batch_timing(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def group_sums1(self, i: int) -> np.ndarray:
        out = np.zeros((BZ_GROUPS, BZ_GROUP_Q1))
        _check(lib().bz_batch_group_sums1(self.h, int(i), out.ctypes.data))
        return out

    def group_sums2(self, i: int, drift) -> np.ndarray:
        d = np.ascontiguousarray(drift, dtype=np.float64)
        out = np.zeros((BZ_GROUPS, BZ_GROUP_Q2))
        _check(lib().bz_batch_group_sums2(self.h, int(i), d.ctypes.data, out.ctypes.data))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().bz_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def step_replay(ctx: Context, mix: Mixture, cfg: bz_swarm_config, state: np.ndarray, ids: np.ndarray,
                steps: np.ndarray, stream=None):
    """One trial step per particle on the GPU (bz_step_replay)."""
    torch = _torch()
    n = int(state.shape[0])
    dev = torch.device("cuda", ctx.device)
    s_in = torch.as_tensor(np.ascontiguousarray(state, np.float64).reshape(-1), device=dev)
    t_ids = torch.as_tensor(np.ascontiguousarray(ids, np.uint64).view(np.int64), device=dev)
    t_steps = torch.as_tensor(np.ascontiguousarray(steps, np.uint32).view(np.int32), device=dev)
    s_out = torch.empty(8 * n, dtype=torch.float64, device=dev)
    dec = torch.empty(n, dtype=torch.int32, device=dev)
    eps = torch.empty(2 * n, dtype=torch.float64, device=dev)
    _check(lib().bz_step_replay(ctx.h, mix.h, C.byref(cfg), n, s_in.data_ptr(), t_ids.data_ptr(),
                                t_steps.data_ptr(), s_out.data_ptr(), dec.data_ptr(), eps.data_ptr(),
                                C.c_void_p(_stream_handle(stream))))
    torch.cuda.synchronize(dev)
    return s_out.cpu().numpy().reshape(n, 8), dec.cpu().numpy(), eps.cpu().numpy().reshape(n, 2)


def philox(ctx: Context, ctr: np.ndarray, key: int, stream=None) -> np.ndarray:
    """Philox4x32-10 of each row of ``ctr`` (n x 4 uint32) on the GPU."""
    torch = _torch()
    dev = torch.device("cuda", ctx.device)
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    n = c.shape[0]
    t_in = torch.as_tensor(c.view(np.int32).reshape(-1), device=dev)
    t_out = torch.empty(4 * n, dtype=torch.int32, device=dev)
    _check(lib().bz_philox(ctx.h, n, t_in.data_ptr(), int(key) & 0xFFFFFFFFFFFFFFFF, t_out.data_ptr(),
                           C.c_void_p(_stream_handle(stream))))
    torch.cuda.synchronize(dev)
    return t_out.cpu().numpy().view(np.uint32).reshape(n, 4)


def run_swarm(ctx: Context, mix: Mixture, cfg: bz_swarm_config, stream=None) -> Swarm:
    return Swarm(ctx, mix, cfg, stream)


def drift_from_group_sums(g1) -> np.ndarray:
    """The swarm's drift vector (6 values) from summed pass-1 group sums (host only)."""
    g = np.ascontiguousarray(g1, dtype=np.float64).reshape(BZ_GROUPS, BZ_GROUP_Q1)
    d = np.zeros(6)
    _check(lib().bz_drift_from_group_sums(g.ctypes.data, d.ctypes.data))
    return d


def finalize_group_sums(g1, g2, e_over_n_Td: float, n_total_m3: float, nu_trial: float = 0.0,
                        n_spawned: int = 0, n_capped: int = 0, error_flags: int = 0) -> Dict[str, float]:
    """Tallies of summed pass-1 and pass-2 group sums (host only)."""
    a = np.ascontiguousarray(g1, dtype=np.float64).reshape(BZ_GROUPS, BZ_GROUP_Q1)
    b = np.ascontiguousarray(g2, dtype=np.float64).reshape(BZ_GROUPS, BZ_GROUP_Q2)
    info = bz_merge_info(float(e_over_n_Td), float(n_total_m3), float(nu_trial), int(n_spawned), int(n_capped),
                         int(error_flags), 0)
    t = bz_tallies()
    _check(lib().bz_finalize_group_sums(a.ctypes.data, b.ctypes.data, C.byref(info), C.byref(t)))
    return _tally_dict(t)
