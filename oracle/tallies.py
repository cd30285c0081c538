"""Swarm estimators of Sec. 2.3 ("Determination of swarm attributes"), FP64.

TEST INFRASTRUCTURE ONLY (part of the oracle).

Input: the per-particle results of a swarm run (final position x, y, z and
time t at the I-th real collision, energy sums, ionization and attachment
counts).  Output: the Drifter quantities of Sec. 7's worked example.

Estimators as the paper writes them (Eqs. 15-27):
  W       = (1/N) sum z_n/t_n                          Eq. (15)/(20)
  alpha   = (1/N) sum G_n/z_n,  eta = (1/N) sum D_n/z_n  Eqs. (16)-(17)
  <eps>   = sum of energies just before each real collision / (N I)   Eq. (18)
  <eps'>  = same, just after                                           Eq. (19)
  d_n     = x_n - t_n W                                 Eq. (21)
  D       = (1/N) sum |d|^2/t,  D_L = (1/N) sum (d.z)^2/(2t),
  D_T     = (1/N) sum |d - (d.z) z|^2/(4t)              Eqs. (22)-(24)
  sigma   = (1/N) sum 2|d|, sigma_L, sigma_T likewise    Eqs. (25)-(27)
  efficiency = real/(real + null + fail)                Eq. (28)
Readings: d_n subtracts the full drift vector W_vec t_n (equal to the paper's
W z-hat t_n whenever the transverse drift vanishes; with B != 0 it keeps the
E x B drift out of D_T); the "d_n - d_n.z" of Eqs. (24) and (27) is read as
the transverse part d - (d.z) z.  mu = W/E, mu N, and the reduced mobility
mu_0 = mu N / N_Loschmidt, as in the worked example of Sec. 7.
Standard errors come from 32 batch groups (particle id mod 32).
"""
from __future__ import annotations

from typing import Dict

import numpy as np

N_LOSCHMIDT = 2.686780111e25  # m^-3, 273.15 K and 101.325 kPa (CODATA 2018)
TOWNSEND = 1e-21


def _estimates(x, y, z, t, sum_e, sum_e2, n_real, n_ion, n_att, W_vec) -> Dict[str, float]:
    dx, dy, dz = x - t * W_vec[0], y - t * W_vec[1], z - t * W_vec[2]
    d2 = dx * dx + dy * dy + dz * dz
    dperp2 = dx * dx + dy * dy
    nr = float(np.sum(n_real))
    return {
        "W": float(np.mean(z / t)),
        "Wx": float(np.mean(x / t)),
        "Wy": float(np.mean(y / t)),
        "alpha": float(np.mean(n_ion / z)),
        "eta": float(np.mean(n_att / z)),
        "eps": float(np.sum(sum_e) / nr) if nr > 0 else 0.0,
        "eps_after": float(np.sum(sum_e2) / nr) if nr > 0 else 0.0,
        "D": float(np.mean(d2 / t)),
        "D_L": float(np.mean(dz * dz / (2.0 * t))),
        "D_T": float(np.mean(dperp2 / (4.0 * t))),
        "sig": float(np.mean(2.0 * np.sqrt(d2))),
        "sig_L": float(np.mean(2.0 * np.abs(dz))),
        "sig_T": float(np.mean(2.0 * np.sqrt(dperp2))),
    }


def swarm_tallies(p: Dict[str, np.ndarray], e_over_n_Td: float, n_total: float, groups: int = 32) -> Dict[str, float]:
    # Eqs. (15)-(27) divide by each particle's time: a particle that never
    # moved (t = 0, e.g. stopped by an error at its first trial) has no
    # defined ratio and is left out
    moved = np.asarray(p["t"], dtype=np.float64) > 0.0
    if not np.all(moved):
        p = {k: (np.asarray(v)[moved] if np.ndim(v) == 1 and len(v) == len(moved) else v) for k, v in p.items()}
    x, y, z, t = (np.asarray(p[k], dtype=np.float64) for k in ("x", "y", "z", "t"))
    sum_e, sum_e2 = np.asarray(p["sum_e"], np.float64), np.asarray(p["sum_e2"], np.float64)
    n_real = np.asarray(p["n_real"], np.float64)
    n_ion, n_att = np.asarray(p["n_ion"], np.float64), np.asarray(p["n_att"], np.float64)
    ids = np.asarray(p["id"], dtype=np.uint64)
    W_vec = np.array([np.mean(x / t), np.mean(y / t), np.mean(z / t)])
    out = _estimates(x, y, z, t, sum_e, sum_e2, n_real, n_ion, n_att, W_vec)
    # batch means: same estimator on each group, with the swarm's drift vector
    g = (ids % groups).astype(np.int64)
    per = {k: [] for k in out}
    for j in range(groups):
        sel = g == j
        if not np.any(sel):
            continue
        e = _estimates(x[sel], y[sel], z[sel], t[sel], sum_e[sel], sum_e2[sel], n_real[sel], n_ion[sel],
                       n_att[sel], W_vec)
        for k, v in e.items():
            per[k].append(v)
    for k, vals in per.items():
        vals = np.asarray(vals)
        out[k + "_se"] = float(np.std(vals, ddof=1) / np.sqrt(len(vals))) if len(vals) > 1 else float("nan")
    # ratio-of-sums forms (flux estimators)
    st = float(np.sum(t))
    Wf = np.array([np.sum(x), np.sum(y), np.sum(z)]) / st
    out["W_flux"] = float(Wf[2])
    out["D_L_flux"] = float(np.sum((z - Wf[2] * t) ** 2) / (2.0 * st))
    out["D_T_flux"] = float(np.sum((x - Wf[0] * t) ** 2 + (y - Wf[1] * t) ** 2) / (4.0 * st))
    out["alpha_flux"] = float(np.sum(n_ion) / np.sum(z))
    out["eta_flux"] = float(np.sum(n_att) / np.sum(z))
    out["lorentz_angle"] = float(np.arctan2(np.hypot(W_vec[0], W_vec[1]), W_vec[2]))
    real, null, fail = (float(np.sum(np.asarray(p[k], np.float64))) for k in ("n_real", "n_null", "n_fail"))
    out["n_real"], out["n_null"], out["n_fail"] = real, null, fail
    out["n_ion"], out["n_att"] = float(np.sum(n_ion)), float(np.sum(n_att))
    out["efficiency"] = real / (real + null + fail) if real + null + fail > 0 else 0.0
    out["n_particles"] = float(len(t))
    out.update(derived(out["W"], out["D"], out["D_L"], out["D_T"], e_over_n_Td, n_total))
    return out


def derived(W: float, D: float, D_L: float, D_T: float, e_over_n_Td: float, n_total: float) -> Dict[str, float]:
    """Mobility and ratio forms printed by the worked example of Sec. 7."""
    E = e_over_n_Td * TOWNSEND * n_total
    mu = W / E if E > 0 else float("nan")
    muN = mu * n_total
    return {
        "E_V_m": E,
        "mu": mu,
        "mu_N": muN,
        "mu_0": muN / N_LOSCHMIDT,
        "D_over_mu": D / mu if mu else float("nan"),
        "D_L_over_mu": D_L / mu if mu else float("nan"),
        "D_T_over_mu": D_T / mu if mu else float("nan"),
        "ND": n_total * D,
    }


def efficiency(real: float, null: float, fail: float) -> float:
    """Eq. (28): real / (real + null + fail)."""
    return real / (real + null + fail)
