"""Seeded synthetic inputs: gases, mixtures, fields and swarm seeds.

This module only builds inputs. It holds none of the transport method's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The paper validates on LXCat cross-section databases (Sec. "Benchmarks") that
are not available here. Every gas below is an invented, deterministic shape
that stands in for the paper's workloads: an Argon-like atom with a
Ramsauer-type dip, three excitations and an ionization; a CO2-like molecule
with vibrational bumps, electronic levels, a dissociative-attachment peak and
an ionization; and a constant-collision-frequency "Maxwell model" gas whose
swarm parameters have closed forms. No value here is a database value.

Channel kinds and angular models use the integer codes of the C interface:
kind 0 elastic, 1 excitation, 2 attachment, 3 ionization; angular model 0
isotropic, 1 screened Coulomb (Sec. "Theoretical framework", Eq.
collision_angle).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# CODATA 2018 exact / recommended values used only to build inputs.
ELEMENTARY_CHARGE = 1.602176634e-19      # C
ELECTRON_MASS = 9.1093837015e-31         # kg
ATOMIC_MASS_UNIT = 1.66053906660e-27     # kg
BOLTZMANN = 1.380649e-23                 # J/K

# Gas number density at 101.325 kPa and 293.15 K, as used by the paper's
# worked drifter example (Sec. "Installation and Usage").
N_STP_293 = 101325.0 / (BOLTZMANN * 293.15)

SEED = 1901081400

ELASTIC, EXCITATION, ATTACHMENT, IONIZATION = 0, 1, 2, 3
ISOTROPIC, SCREENED_COULOMB, XI_FORM = 0, 1, 2


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014); used only to derive seeds."""
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def swarm_seed(index: int, base: int = SEED) -> int:
    """Philox key of swarm ``index`` derived from the base seed."""
    return splitmix64((base * 0x100000001B3 + index) & 0xFFFFFFFFFFFFFFFF)


@dataclasses.dataclass
class Channel:
    kind: int
    threshold_eV: float
    energy_eV: np.ndarray
    sigma_m2: np.ndarray


@dataclasses.dataclass
class Gas:
    name: str
    mass_kg: float
    number_density_m3: float
    angular: int
    channels: List[Channel]
    # XI_FORM gases: the total elastic cross section (energy [eV], sigma [m^2]);
    # the elastic channel's table is the momentum-transfer cross section
    sigma_el: Optional[Tuple[np.ndarray, np.ndarray]] = None

    def with_density(self, n: float) -> "Gas":
        return dataclasses.replace(self, number_density_m3=float(n))


@dataclasses.dataclass
class SwarmSpec:
    """One swarm of a workload: which gases, the fields and the run sizes."""
    gases: List[Gas]
    e_over_n_Td: float
    b_T: float
    b_angle_rad: float
    n_electrons: int
    real_collisions: int
    seed: int
    precision: int = 32
    eps0_mean_eV: float = 0.1


def _loglog_through(anchors: Sequence[tuple], energies: np.ndarray) -> np.ndarray:
    le = np.log([a[0] for a in anchors])
    ls = np.log([a[1] for a in anchors])
    return np.exp(np.interp(np.log(energies), le, ls))


# --------------------------------------------------------------------------
# Maxwell model: one elastic channel with a constant collision frequency.
# --------------------------------------------------------------------------
def maxwell_gas(nu: float = 1e12, mass_ratio: float = 1e-4, n: float = N_STP_293,
                points: int = 2001, e_lo: float = 1e-4, e_hi: float = 1e4) -> Gas:
    """Elastic sigma proportional to 1/v so that nu = n sigma v is constant.

    Tabulated on ``points`` log-spaced energies; m/M = ``mass_ratio``.
    """
    e = np.geomspace(e_lo, e_hi, points)
    speed = np.sqrt(2.0 * e * ELEMENTARY_CHARGE / ELECTRON_MASS)
    sigma = nu / (n * speed)
    ch = Channel(ELASTIC, 0.0, e, sigma)
    return Gas("maxwell", ELECTRON_MASS / mass_ratio, n, ISOTROPIC, [ch])


# --------------------------------------------------------------------------
# Argon-like atom.
# --------------------------------------------------------------------------
def _ramp_then_flat(th: float, peak: float, rise: float = 5.0, top: float = 100.0,
                    n_rise: int = 10, n_total: int = 40) -> Channel:
    e_rise = np.linspace(th, th + rise, n_rise)
    e_flat = np.geomspace(th + rise, top, n_total - n_rise + 1)[1:]
    e = np.concatenate([e_rise, e_flat])
    s = np.where(e <= th + rise, peak * (e - th) / rise, peak)
    s[0] = 0.0
    return Channel(EXCITATION, th, e, s)


def argon_like(n: float = N_STP_293) -> Gas:
    """Elastic sigma_m with a Ramsauer-type dip, 3 excitations, 1 ionization."""
    e_el = np.geomspace(1e-3, 100.0, 200)
    s_el = _loglog_through([(1e-3, 6e-20), (0.25, 1e-21), (12.0, 1.5e-19), (100.0, 4e-20)], e_el)
    chans = [Channel(ELASTIC, 0.0, e_el, s_el)]
    for th in (11.5, 11.8, 13.0):
        chans.append(_ramp_then_flat(th, 1e-21))
    ip = 15.76
    e_io = np.linspace(ip, 100.0, 40)
    s_io = 2.5e-20 * (e_io - ip) / (100.0 - ip)
    chans.append(Channel(IONIZATION, ip, e_io, s_io))
    return Gas("argon-like", 39.948 * ATOMIC_MASS_UNIT, n, ISOTROPIC, chans)


# --------------------------------------------------------------------------
# CO2-like molecule (20 channels on 500-point log tables).
# --------------------------------------------------------------------------
def _triangle(e: np.ndarray, th: float, peak: float, width: float) -> np.ndarray:
    up = (e - th) / width
    down = (th + 3.0 * width - e) / (2.0 * width)
    return peak * np.clip(np.minimum(up, down), 0.0, None)


def _on_grid(grid: np.ndarray, th: float, lo: float = 0.0, hi: float = np.inf) -> np.ndarray:
    """Energies of an inelastic table on a gas's common grid: the threshold,
    then the grid points above it (inside [lo, hi])."""
    pts = grid[(grid > th) & (grid >= lo) & (grid <= hi)]
    return np.concatenate([[th], pts])


def co2_like(n: float = N_STP_293, points: int = 500, xi_form: bool = False) -> Gas:
    """20 channels; every table lives on the gas's 500-point log grid
    (1e-3 - 100 eV), inelastic ones from their threshold upwards.  With
    xi_form the gas scatters by the xi form of a non-polar molecule, with a
    total elastic cross section sigma_el = sigma_mt (1 + eps / 5 eV), so
    that scattering turns forward as the energy grows."""
    grid = np.geomspace(1e-3, 100.0, points)
    s_el = 1e-20 + 9e-20 / (1.0 + (grid / 0.5) ** 0.8)
    chans = [Channel(ELASTIC, 0.0, grid, s_el)]
    for th in np.geomspace(0.083, 2.5, 8):
        e = _on_grid(grid, float(th))
        s = _triangle(e, th, 2e-21, max(0.3 * th, 0.05))
        s[0] = 0.0
        chans.append(Channel(EXCITATION, float(th), e, s))
    for th in np.linspace(7.0, 13.0, 9):
        e = _on_grid(grid, float(th))
        s = np.where(e <= th + 5.0, 5e-22 * (e - th) / 5.0, 5e-22)
        s[0] = 0.0
        chans.append(Channel(EXCITATION, float(th), e, s))
    # dissociative attachment: Gaussian peak at 4.4 eV, zero outside 3-6 eV
    e = np.concatenate([_on_grid(grid, 3.0, hi=6.0), [6.0, 100.0]])
    s = 1.5e-22 * np.exp(-0.5 * ((e - 4.4) / 0.5) ** 2)
    s[0] = 0.0
    s[-2:] = 0.0
    chans.append(Channel(ATTACHMENT, 3.0, e, s))
    ip = 13.8
    e = _on_grid(grid, ip)
    s = 2e-20 * (e - ip) / (100.0 - ip)
    chans.append(Channel(IONIZATION, ip, e, s))
    if xi_form:
        return Gas("co2-like-xi", 44.01 * ATOMIC_MASS_UNIT, n, XI_FORM, chans,
                   sigma_el=(grid.copy(), s_el * (1.0 + grid / 5.0)))
    return Gas("co2-like", 44.01 * ATOMIC_MASS_UNIT, n, ISOTROPIC, chans)


# --------------------------------------------------------------------------
# Random gases for the batched workload.
# --------------------------------------------------------------------------
def random_gas(rng: np.random.Generator, name: str, n: float = N_STP_293) -> Gas:
    """1 elastic + a random mix of vibrational, electronic, attachment and
    ionization channels shaped like the Argon-like and CO2-like gases."""
    points = int(rng.integers(100, 1001))
    n_ch = int(rng.integers(5, 41))
    mass = float(rng.uniform(4.0, 150.0)) * ATOMIC_MASS_UNIT
    e_el = np.geomspace(1e-3, 100.0, points)
    dip_e = float(np.exp(rng.uniform(np.log(0.05), np.log(2.0))))
    anchors = [(1e-3, float(rng.uniform(5e-21, 8e-20))), (dip_e, float(rng.uniform(5e-22, 5e-21))),
               (float(rng.uniform(5.0, 20.0)), float(rng.uniform(5e-20, 2e-19))), (100.0, float(rng.uniform(2e-20, 6e-20)))]
    anchors.sort()
    chans = [Channel(ELASTIC, 0.0, e_el, _loglog_through(anchors, e_el))]
    has_ion = False
    has_att = False
    for _ in range(n_ch - 1):
        pick = rng.uniform()
        if pick < 0.45:
            th = float(np.exp(rng.uniform(np.log(0.05), np.log(3.0))))
            e = _on_grid(e_el, th)
            s = _triangle(e, th, float(rng.uniform(5e-22, 3e-21)), max(0.3 * th, 0.05))
        elif pick < 0.85 or has_ion:
            th = float(rng.uniform(6.0, 15.0))
            e = _on_grid(e_el, th)
            peak = float(rng.uniform(1e-22, 1e-21))
            s = np.where(e <= th + 5.0, peak * (e - th) / 5.0, peak)
        elif pick < 0.93 and not has_att:
            has_att = True
            c = float(rng.uniform(2.0, 8.0))
            e = np.concatenate([_on_grid(e_el, c - 1.5, hi=c + 1.5), [c + 1.5, 100.0]])
            s = float(rng.uniform(5e-23, 3e-22)) * np.exp(-0.5 * ((e - c) / 0.5) ** 2)
            s[0] = 0.0
            s[-2:] = 0.0
            chans.append(Channel(ATTACHMENT, c - 1.5, e, s))
            continue
        else:
            has_ion = True
            th = float(rng.uniform(10.0, 25.0))
            e = _on_grid(e_el, th)
            s = float(rng.uniform(1e-20, 4e-20)) * (e - th) / (100.0 - th)
            s[0] = 0.0
            chans.append(Channel(IONIZATION, th, e, s))
            continue
        s = np.asarray(s, dtype=np.float64)
        s[0] = 0.0
        chans.append(Channel(EXCITATION, th, e, s))
    return Gas(name, mass, n, ISOTROPIC, chans)


def batched_gases(seed: int = SEED) -> List[Gas]:
    rng = np.random.default_rng(splitmix64(seed ^ 0xB47C4ED))
    return [random_gas(rng, f"synthetic-{i}") for i in range(8)]


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
def maxwell_swarm(n_electrons: int = 10_000, real_collisions: int = 1000, index: int = 0) -> SwarmSpec:
    """Maxwell-model gas, E/N = 10 Td, B = 0, FP64, Maxwellian start, mean 0.1 eV."""
    return SwarmSpec([maxwell_gas()], 10.0, 0.0, 0.0, n_electrons, real_collisions,
                     swarm_seed(index), precision=64, eps0_mean_eV=0.1)


def argon_sweep_fields(points: int = 32) -> np.ndarray:
    """E/N values of the Argon-like sweep: 1 to 1000 Td, log-spaced."""
    return np.geomspace(1.0, 1000.0, points)


def argon_sweep(n_electrons: int = 1_000_000, real_collisions: int = 1000,
                points: int = 32) -> List[SwarmSpec]:
    gas = argon_like()
    return [SwarmSpec([gas], float(f), 0.0, 0.0, n_electrons, real_collisions,
                      swarm_seed(1000 + i), precision=32)
            for i, f in enumerate(argon_sweep_fields(points))]


def ar_co2_mixture(n_total: float = N_STP_293) -> List[Gas]:
    return [argon_like(0.9 * n_total), co2_like(0.1 * n_total)]


def ar_co2_avalanche_mixture(n_total: float = N_STP_293) -> List[Gas]:
    """Ar/CO2 93/7, the mixture of the paper's avalanche timing (Sec. 8)."""
    return [argon_like(0.93 * n_total), co2_like(0.07 * n_total)]


def ar_co2_swarm(n_electrons: int = 1_000_000, real_collisions: int = 1000) -> SwarmSpec:
    """Ar/CO2 90/10, E/N = 100 Td, B = 1 T perpendicular to E."""
    return SwarmSpec(ar_co2_mixture(), 100.0, 1.0, math.pi / 2, n_electrons, real_collisions,
                     swarm_seed(2000), precision=32)


def batched_swarms(count: int = 256, real_collisions: int = 1000, seed: int = SEED,
                   max_electrons: int = 1_000_000) -> List[SwarmSpec]:
    """256 swarms: n_e log-uniform 1e3-1e6, 2-4 gases with Dirichlet(1)
    fractions, E/N log-uniform 0.1-1000 Td, |B| uniform 0-2 T, cos(theta_B)
    uniform in [-1, 1]."""
    gases = batched_gases(seed)
    rng = np.random.default_rng(splitmix64(seed ^ 0x5A55A5))
    out = []
    for i in range(count):
        k = int(rng.integers(2, 5))
        pick = rng.choice(len(gases), size=k, replace=False)
        frac = rng.dirichlet(np.ones(k))
        mix = [gases[j].with_density(f * N_STP_293) for j, f in zip(pick, frac)]
        n_e = int(round(math.exp(rng.uniform(math.log(1e3), math.log(max_electrons)))))
        eon = float(math.exp(rng.uniform(math.log(0.1), math.log(1000.0))))
        b = float(rng.uniform(0.0, 2.0))
        ang = float(math.acos(rng.uniform(-1.0, 1.0)))
        out.append(SwarmSpec(mix, eon, b, ang, n_e, real_collisions, swarm_seed(3000 + i)))
    return out


def flatten_gases(gases: Sequence[Gas]):
    """Flat arrays of a mixture, in the order the C interfaces take them.

    Returns a dict with per-gas arrays (mass, density, angular, first channel,
    channel count) and per-channel arrays (gas, kind, threshold, offset, n)
    plus the concatenated energy and sigma tables (float64).
    """
    g_mass, g_dens, g_ang, g_first, g_nch = [], [], [], [], []
    c_gas, c_kind, c_th, c_off, c_n = [], [], [], [], []
    e_all, s_all = [], []
    el_off, el_n, el_e, el_s = [], [], [], []
    off = 0
    el_at = 0
    for gi, g in enumerate(gases):
        g_mass.append(g.mass_kg)
        g_dens.append(g.number_density_m3)
        g_ang.append(g.angular)
        g_first.append(len(c_gas))
        g_nch.append(len(g.channels))
        if g.sigma_el is not None:
            ee = np.ascontiguousarray(g.sigma_el[0], dtype=np.float64)
            ss = np.ascontiguousarray(g.sigma_el[1], dtype=np.float64)
            el_off.append(el_at)
            el_n.append(len(ee))
            el_e.append(ee)
            el_s.append(ss)
            el_at += len(ee)
        else:
            el_off.append(el_at)
            el_n.append(0)
        for ch in g.channels:
            e = np.ascontiguousarray(ch.energy_eV, dtype=np.float64)
            s = np.ascontiguousarray(ch.sigma_m2, dtype=np.float64)
            c_gas.append(gi)
            c_kind.append(ch.kind)
            c_th.append(ch.threshold_eV)
            c_off.append(off)
            c_n.append(len(e))
            e_all.append(e)
            s_all.append(s)
            off += len(e)
    return dict(
        gas_mass=np.array(g_mass, dtype=np.float64), gas_density=np.array(g_dens, dtype=np.float64),
        gas_angular=np.array(g_ang, dtype=np.int32), gas_first=np.array(g_first, dtype=np.int32),
        gas_nch=np.array(g_nch, dtype=np.int32),
        ch_gas=np.array(c_gas, dtype=np.int32), ch_kind=np.array(c_kind, dtype=np.int32),
        ch_threshold=np.array(c_th, dtype=np.float64), ch_offset=np.array(c_off, dtype=np.int64),
        ch_n=np.array(c_n, dtype=np.int32),
        energy=np.concatenate(e_all) if e_all else np.zeros(0),
        sigma=np.concatenate(s_all) if s_all else np.zeros(0),
        gas_el_offset=np.array(el_off, dtype=np.int64), gas_el_n=np.array(el_n, dtype=np.int32),
        el_energy=np.concatenate(el_e) if el_e else np.zeros(1), el_sigma=np.concatenate(el_s) if el_s else np.zeros(1),
    )
