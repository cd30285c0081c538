"""ctypes wrapper of the FP64 oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it; the product path never does.

Parity status of the oracle's functions (each pinned by a ``-m "not gpu"``
test against something other than itself):
  philox / uniform      known answers of cuRAND's host Philox4_32_10
                        generator; uniformity, independence, avalanche
  sigma (tables+ext.)   hand-worked cases of Sec. 2.2, Eqs. (12)-(14)
  nu, select_channel    Eq. (2) against channel ratios (chi-square)
  majorant              brute-force maximum on a dense grid
  cos_theta             closed-form <1 - cos> of Eq. (5), isotropic moments
  ratio_elastic/inel.   exact two-body kinematics in the centre-of-mass frame
  rotate                orthonormality and the prescribed polar angle
  move                  brute-force RK4 integration of the Lorentz force
  run_swarm             closed forms of the constant-frequency Maxwell model
                        (drift velocity, mean energy, D_L, D_T)
  ionization split      closed-form moments of one ionizing collision (Eq. 9
                        with the uniform split of the remaining energy): mean,
                        second moment, correlation with the scattering cosine
  dummy attachment      the reading of Sec. 2 (a plastic collision: the
                        electron stops), checked directly
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Sequence

import numpy as np

from . import build as _build

_lib = None

DEC_FAIL, DEC_NULL = -2, -1
ST_DONE, ST_TIME, ST_STEPS, ST_TRIAL, ST_ERROR, ST_ATTACHED = 0, 1, 2, 3, 4, 5

_dp = C.POINTER(C.c_double)
_u32p = C.POINTER(C.c_uint32)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_u64p = C.POINTER(C.c_uint64)


class _Config(C.Structure):
    _fields_ = [("e_over_n_Td", C.c_double), ("b_T", C.c_double), ("b_angle_rad", C.c_double),
                ("nu_trial", C.c_double), ("fixed", C.c_int), ("real_collisions", C.c_uint32),
                ("t_end", C.c_double), ("eps0_mean_eV", C.c_double), ("seed", C.c_uint64),
                ("max_trials", C.c_uint64), ("attach_keep_state", C.c_int), ("spawn", C.c_int),
                ("pop_cap", C.c_uint64), ("strategy", C.c_int), ("zeta", C.c_double), ("grace", C.c_uint32),
                ("bins_per_decade", C.c_int), ("gas_T", C.c_double)]


# trial frequency strategies of Sec. 6 (besides the constant one)
TF_CONST, TF_VARIABLE, TF_BINNED = 0, 1, 2


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.or_uniform.restype = C.c_double
        L.or_uniform.argtypes = [C.c_uint32]
        L.or_mixture_create.restype = C.c_int
        L.or_mixture_create.argtypes = [C.c_int, _dp, _dp, _i32p, C.c_int, _i32p, _i32p, _dp, _i64p, _i32p,
                                        _dp, _dp, _i64p, _i32p, _dp, _dp, C.c_double, C.POINTER(C.c_void_p)]
        L.or_xi_ratio.restype = C.c_double
        L.or_xi_ratio.argtypes = [C.c_double]
        L.or_xi_solve.restype = C.c_double
        L.or_xi_solve.argtypes = [C.c_double]
        L.or_cos_theta_xi.restype = C.c_double
        L.or_cos_theta_xi.argtypes = [C.c_double, C.c_double]
        L.or_gas_xi.restype = C.c_double
        L.or_gas_xi.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.or_mixture_destroy.argtypes = [C.c_void_p]
        for f in ("or_mixture_nu_max", "or_mixture_eps_at_max", "or_mixture_n_total"):
            getattr(L, f).restype = C.c_double
            getattr(L, f).argtypes = [C.c_void_p]
        L.or_sigma.restype = C.c_double
        L.or_sigma.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.or_nu.restype = C.c_double
        L.or_nu.argtypes = [C.c_void_p, C.c_double]
        L.or_density_sum.restype = C.c_double
        L.or_density_sum.argtypes = [C.c_void_p, C.c_double]
        L.or_select_channel.restype = C.c_int
        L.or_select_channel.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.or_cos_theta.restype = C.c_double
        L.or_cos_theta.argtypes = [C.c_int, C.c_double, C.c_double]
        L.or_ratio_elastic.restype = C.c_double
        L.or_ratio_elastic.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_ratio_inelastic.restype = C.c_double
        L.or_ratio_inelastic.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_rotate.argtypes = [_dp, C.c_double, C.c_double, _dp]
        L.or_move_flat.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, _dp, _dp, C.c_double]
        L.or_run_swarm.restype = C.c_int
        L.or_run_swarm.argtypes = [C.c_void_p, C.POINTER(_Config), C.c_uint64, C.c_int64, C.c_int] + \
            [_dp] * 10 + [_u32p] * 7
        L.or_step_replay.restype = C.c_int
        L.or_step_replay.argtypes = [C.c_void_p, C.POINTER(_Config), C.c_int64, _dp, _u64p, _u32p, _dp, _i32p, _dp]
        L.or_initial_velocity.argtypes = [C.c_double, C.c_uint64, C.c_uint64, _dp]
        L.or_nu_many.argtypes = [C.c_void_p, C.c_int64, _dp, _dp]
        L.or_secondary_id.restype = C.c_uint64
        L.or_secondary_id.argtypes = [C.c_uint64, C.c_uint32]
        L.or_run_swarm_spawn.restype = C.c_int64
        L.or_run_swarm_spawn.argtypes = [C.c_void_p, C.POINTER(_Config), C.c_uint64, C.c_int64, C.c_int64] + \
            [_dp] * 10 + [_u32p] * 7 + [_u64p, _dp]
        L.or_sigma_many.argtypes = [C.c_void_p, C.c_int, C.c_int64, _dp, _dp]
        L.or_initial_velocity_many.argtypes = [C.c_double, C.c_uint64, C.c_uint64, C.c_int64, _dp]
        L.or_thermal_collide.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                         _dp, _dp]
        L.or_range_max.restype = C.c_double
        L.or_range_max.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.or_binned_max.restype = C.c_double
        L.or_binned_max.argtypes = [C.c_void_p, C.c_int, C.c_int]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


# -------------------------------------------------------------------------
def philox(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(o, _u32p))
    return o


def uniform(w: int) -> float:
    return lib().or_uniform(int(w) & 0xFFFFFFFF)


class Mixture:
    """Gas mixture held by the oracle (tables copied as given)."""

    def __init__(self, gases, eps_cap: float = 0.0):
        from paper_1901_08140_gb300.workloads import flatten_gases
        f = flatten_gases(gases)
        self._keep = f
        h = C.c_void_p()
        rc = lib().or_mixture_create(len(f["gas_mass"]), _p(f["gas_mass"], _dp), _p(f["gas_density"], _dp),
                                     _p(f["gas_angular"], _i32p), len(f["ch_gas"]), _p(f["ch_gas"], _i32p),
                                     _p(f["ch_kind"], _i32p), _p(f["ch_threshold"], _dp), _p(f["ch_offset"], _i64p),
                                     _p(f["ch_n"], _i32p), _p(f["energy"], _dp), _p(f["sigma"], _dp),
                                     _p(f["gas_el_offset"], _i64p), _p(f["gas_el_n"], _i32p),
                                     _p(f["el_energy"], _dp), _p(f["el_sigma"], _dp), float(eps_cap), C.byref(h))
        if rc != 0:
            raise ValueError("oracle rejected the mixture")
        self.h = h
        self.n_channels = len(f["ch_gas"])
        self.ch_kind = f["ch_kind"]
        self.ch_gas = f["ch_gas"]
        self.ch_threshold = f["ch_threshold"]
        self.gas_mass = f["gas_mass"]
        self.gas_density = f["gas_density"]
        self.gas_angular = f["gas_angular"]

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.or_mixture_destroy(self.h)
            self.h = None

    @property
    def nu_max(self) -> float:
        return lib().or_mixture_nu_max(self.h)

    @property
    def eps_at_max(self) -> float:
        return lib().or_mixture_eps_at_max(self.h)

    @property
    def n_total(self) -> float:
        return lib().or_mixture_n_total(self.h)

    def sigma(self, c: int, eps: float) -> float:
        return lib().or_sigma(self.h, int(c), float(eps))

    def nu(self, eps: float) -> float:
        return lib().or_nu(self.h, float(eps))

    def nu_many(self, eps) -> np.ndarray:
        e = np.ascontiguousarray(eps, dtype=np.float64)
        o = np.zeros_like(e)
        lib().or_nu_many(self.h, e.size, _p(e, _dp), _p(o, _dp))
        return o

    def sigma_many(self, c: int, eps) -> np.ndarray:
        e = np.ascontiguousarray(eps, dtype=np.float64)
        o = np.zeros_like(e)
        lib().or_sigma_many(self.h, int(c), e.size, _p(e, _dp), _p(o, _dp))
        return o

    def density_sum(self, eps: float) -> float:
        return lib().or_density_sum(self.h, float(eps))

    def select_channel(self, eps: float, r: float) -> int:
        return lib().or_select_channel(self.h, float(eps), float(r))

    def gas_xi(self, g: int, eps: float) -> float:
        """xi of gas g at eps (Eq. 7) from sigma_mt / sigma_el."""
        return lib().or_gas_xi(self.h, int(g), float(eps))

    def range_max(self, a: float, b: float) -> float:
        """Maximum of nu over [a, b] eV."""
        return lib().or_range_max(self.h, float(a), float(b))

    def binned_max(self, bins_per_decade: int, j: int) -> float:
        """Maximum of nu over bin j = [10^(j/B), 10^((j+1)/B)) (BinnedTrialFrequency)."""
        return lib().or_binned_max(self.h, int(bins_per_decade), int(j))


def cos_theta(angular: int, eps_eV: float, R: float) -> float:
    return lib().or_cos_theta(int(angular), float(eps_eV), float(R))


def thermal_collide(v1, v2, m: float, M: float, eps_k: float, cos_t: float, phi: float):
    """One collision with a moving target in the centre-of-momentum frame (Sec. 2.1)."""
    a = np.ascontiguousarray(v1, dtype=np.float64)
    b = np.ascontiguousarray(v2, dtype=np.float64)
    o1, o2 = np.zeros(3), np.zeros(3)
    lib().or_thermal_collide(_p(a, _dp), _p(b, _dp), float(m), float(M), float(eps_k), float(cos_t), float(phi),
                             _p(o1, _dp), _p(o2, _dp))
    return o1, o2


def xi_ratio(xi: float) -> float:
    """sigma_mt / sigma_el produced by the xi form (right side of Eq. 7)."""
    return lib().or_xi_ratio(float(xi))


def xi_solve(r: float) -> float:
    return lib().or_xi_solve(float(r))


def cos_theta_xi(xi: float, R: float) -> float:
    return lib().or_cos_theta_xi(float(xi), float(R))


def ratio_elastic(m: float, M: float, cos_t: float) -> float:
    return lib().or_ratio_elastic(m, M, cos_t)


def ratio_inelastic(m: float, M: float, eps_i: float, eps_k: float, cos_t: float) -> float:
    return lib().or_ratio_inelastic(m, M, eps_i, eps_k, cos_t)


def rotate(d, cos_t: float, phi: float) -> np.ndarray:
    d = np.ascontiguousarray(d, dtype=np.float64)
    o = np.zeros(3)
    lib().or_rotate(_p(d, _dp), float(cos_t), float(phi), _p(o, _dp))
    return o


def move(x, v, dt: float, e_over_n_Td: float, n_total: float, b_T: float = 0.0, b_angle_rad: float = 0.0):
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    lib().or_move_flat(e_over_n_Td, n_total, b_T, b_angle_rad, _p(x, _dp), _p(v, _dp), float(dt))
    return x, v


def initial_velocity(eps0_mean_eV: float, seed: int, pid: int) -> np.ndarray:
    o = np.zeros(3)
    lib().or_initial_velocity(float(eps0_mean_eV), int(seed), int(pid), _p(o, _dp))
    return o


def initial_velocities(eps0_mean_eV: float, seed: int, id0: int, n: int) -> np.ndarray:
    o = np.zeros((n, 3))
    lib().or_initial_velocity_many(float(eps0_mean_eV), int(seed), int(id0), int(n), _p(o, _dp))
    return o


def _config(e_over_n_Td, b_T, b_angle_rad, real_collisions, seed, eps0_mean_eV, nu_trial, fixed, t_end,
            max_trials, attach_keep_state, spawn=False, pop_cap=0, strategy=TF_CONST, zeta=0.25, grace=5000,
            bins_per_decade=8, gas_T=0.0) -> _Config:
    return _Config(float(e_over_n_Td), float(b_T), float(b_angle_rad), float(nu_trial), int(bool(fixed)),
                   int(real_collisions), float(t_end), float(eps0_mean_eV), int(seed) & 0xFFFFFFFFFFFFFFFF,
                   int(max_trials), int(bool(attach_keep_state)), int(bool(spawn)), int(pop_cap), int(strategy),
                   float(zeta), int(grace), int(bins_per_decade), float(gas_T))


def secondary_id(parent: int, step: int) -> int:
    return lib().or_secondary_id(int(parent), int(step))


def run_swarm_spawn(mix: Mixture, *, e_over_n_Td: float, real_collisions: int, n: int, seed: int, pop_cap: int,
                    b_T: float = 0.0, b_angle_rad: float = 0.0, id0: int = 0, eps0_mean_eV: float = 0.1,
                    nu_trial: float = 0.0, t_end: float = 0.0, max_trials: int = 0,
                    **strategy) -> Dict[str, np.ndarray]:
    """Spawn mode: ionizations create electrons, attachments remove them.
    ``strategy``: strategy=TF_VARIABLE | TF_BINNED with zeta, grace, bins_per_decade."""
    cf = _config(e_over_n_Td, b_T, b_angle_rad, real_collisions, seed, eps0_mean_eV, nu_trial, False, t_end,
                 max_trials, False, spawn=True, pop_cap=pop_cap, **strategy)
    names_d = ["x", "y", "z", "t", "vx", "vy", "vz", "sum_e", "sum_e2", "nu_p"]
    names_u = ["n_real", "n_null", "n_fail", "n_ion", "n_att", "steps", "status"]
    out = {k: np.zeros(pop_cap, dtype=np.float64) for k in names_d}
    out.update({k: np.zeros(pop_cap, dtype=np.uint32) for k in names_u})
    ids = np.zeros(pop_cap, dtype=np.uint64)
    tb = np.zeros(pop_cap, dtype=np.float64)
    total = lib().or_run_swarm_spawn(mix.h, C.byref(cf), int(id0), int(n), int(pop_cap),
                                     *[_p(out[k], _dp) for k in names_d], *[_p(out[k], _u32p) for k in names_u],
                                     _p(ids, _u64p), _p(tb, _dp))
    if total == -1:
        raise ValueError("pop_cap below the number of primaries")
    if total < 0:
        raise ValueError("invalid trial frequency strategy")
    res = {k: v[:total] for k, v in out.items()}
    res["id"] = ids[:total]
    res["t_birth"] = tb[:total]
    return res


def run_swarm(mix: Mixture, *, e_over_n_Td: float, real_collisions: int, n: int, seed: int,
              b_T: float = 0.0, b_angle_rad: float = 0.0, id0: int = 0, eps0_mean_eV: float = 0.1,
              nu_trial: float = 0.0, fixed: bool = False, t_end: float = 0.0, threads: int = 1,
              max_trials: int = 0, attach_keep_state: bool = False, **strategy) -> Dict[str, np.ndarray]:
    """Runs particles id0..id0+n-1 to I real collisions; per-particle outputs.
    ``strategy``: strategy=TF_VARIABLE | TF_BINNED with zeta, grace, bins_per_decade (Sec. 6)."""
    cf = _config(e_over_n_Td, b_T, b_angle_rad, real_collisions, seed, eps0_mean_eV, nu_trial, fixed, t_end,
                 max_trials, attach_keep_state, **strategy)
    names_d = ["x", "y", "z", "t", "vx", "vy", "vz", "sum_e", "sum_e2", "nu_p"]
    names_u = ["n_real", "n_null", "n_fail", "n_ion", "n_att", "steps", "status"]
    out = {k: np.zeros(n, dtype=np.float64) for k in names_d}
    out.update({k: np.zeros(n, dtype=np.uint32) for k in names_u})
    if n == 0:
        out["id"] = np.zeros(0, dtype=np.uint64)
        return out
    rc = lib().or_run_swarm(mix.h, C.byref(cf), int(id0), int(n), int(threads),
                            *[_p(out[k], _dp) for k in names_d], *[_p(out[k], _u32p) for k in names_u])
    if rc != 0:
        raise ValueError("invalid trial frequency strategy")
    out["id"] = np.arange(id0, id0 + n, dtype=np.uint64)
    return out


def step_replay(mix: Mixture, state: np.ndarray, ids: np.ndarray, steps: np.ndarray, *, e_over_n_Td: float,
                seed: int, b_T: float = 0.0, b_angle_rad: float = 0.0, attach_keep_state: bool = False):
    """One trial step per particle from ``state`` (n x 8: x, y, z, vx, vy, vz, t, nu')."""
    state = np.ascontiguousarray(state, dtype=np.float64)
    n = state.shape[0]
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    steps = np.ascontiguousarray(steps, dtype=np.uint32)
    cf = _config(e_over_n_Td, b_T, b_angle_rad, 1, seed, 0.0, 0.0, False, 0.0, 0, attach_keep_state)
    out = np.zeros_like(state)
    dec = np.zeros(n, dtype=np.int32)
    eps = np.zeros(2 * n, dtype=np.float64)
    lib().or_step_replay(mix.h, C.byref(cf), n, _p(state, _dp), _p(ids, _u64p), _p(steps, _u32p),
                         _p(out, _dp), _p(dec, _i32p), _p(eps, _dp))
    return out, dec, eps.reshape(n, 2)


def cpu_count() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:  # pragma: no cover
        return os.cpu_count() or 1
