"""Moving targets (Sec. 2.1) on the GPU: against the FP64 oracle electron by
electron, and against the closed forms of a constant-frequency gas."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import tallies as OT
from paper_1901_08140_gb300 import bz
from paper_1901_08140_gb300 import workloads as W

pytestmark = pytest.mark.gpu

QE = 1.602176634e-19
ME = 9.1093837015e-31
KB = 1.380649e-23


@pytest.fixture(scope="module")
def ctx():
    from paper_1901_08140_gb300 import build as B
    B.build()
    c = bz.Context(0)
    yield c
    c.close()


def _gpu(ctx, gases, **kw):
    mix = bz.Mixture(ctx, gases)
    sw = bz.run_swarm(ctx, mix, bz.make_config(**kw))
    t = sw.tallies()
    p = sw.particles()
    sw.close()
    return t, p


def test_fp64_matches_the_oracle_electron_by_electron(ctx):
    gases = W.ar_co2_mixture()
    kw = dict(e_over_n_Td=10.0, real_collisions=300, seed=71)
    t, p = _gpu(ctx, gases, n_electrons=2000, precision=64, gas_temperature_K=293.15, **kw)
    po = O.run_swarm(O.Mixture(gases), n=2000, threads=O.cpu_count(), gas_T=293.15, **kw)
    same = np.ones(2000, bool)
    for k in ["n_real", "n_null", "n_fail", "n_ion", "n_att", "steps", "status"]:
        same &= p[k] == po[k]
    assert same.mean() > 0.99
    for k in ["z", "t", "sum_e"]:
        scale = np.abs(po[k][same]) + 1e-6 * np.abs(po[k]).mean()
        assert np.all(np.abs(p[k][same] - po[k][same]) / scale < 1e-8), k


def test_constant_frequency_closed_forms_fp32(ctx):
    """v_d = eE/(mu nu) and <eps> = 3/2 kT + (eE)^2/(mu nu^2 kappa) for a light
    target (M = 10 m), constant nu, isotropic scattering -- compared as the
    exact means of the run from its start (the transient of the first few
    collisions included), on the ratio-of-sums drift and the
    collision-averaged energy."""
    from test_oracle_pins import thermal_expectations
    temp, nu = 293.15, 1e12
    gas = W.maxwell_gas(nu=nu, mass_ratio=0.1)
    eon = 10.0
    E = eon * 1e-21 * gas.number_density_m3
    w_exp, e_exp = thermal_expectations(1000, 0.1, nu, E, gas.mass_kg, temp)
    for mode in (bz.BZ_TRIAL_LAZY, bz.BZ_TRIAL_WINDOW):
        t, _ = _gpu(ctx, [gas], n_electrons=200000, real_collisions=1000, e_over_n_Td=eon, seed=72, precision=32,
                    trial_mode=mode, gas_temperature_K=temp)
        assert abs(t["W_flux"] - w_exp) < 3.5 * t["W_se"], (mode, t["W_flux"], w_exp, t["W_se"])
        assert abs(t["eps"] - e_exp) < 3.5 * t["eps_se"], (mode, t["eps"], e_exp, t["eps_se"])


def test_equilibrium_at_zero_field(ctx):
    temp = 293.15
    kT = KB * temp / QE
    gas = W.maxwell_gas(nu=1e12, mass_ratio=0.1)
    _, p = _gpu(ctx, [gas], n_electrons=100000, real_collisions=300, e_over_n_Td=0.0, seed=73, precision=32,
                gas_temperature_K=temp)
    eps = 0.5 * ME * (p["vx"].astype(np.float64) ** 2 + p["vy"] ** 2 + p["vz"] ** 2) / QE
    assert abs(eps.mean() - 1.5 * kT) < 4 * eps.std() / math.sqrt(len(eps))


def test_invalid_temperature(ctx):
    mix = bz.Mixture(ctx, [W.argon_like()])
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(bz.BzError):
            bz.run_swarm(ctx, mix, bz.make_config(n_electrons=10, real_collisions=10, e_over_n_Td=10.0,
                                                  gas_temperature_K=bad))
