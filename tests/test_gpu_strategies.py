"""The paper's adaptive trial frequencies (Sec. 6.3 Binned, Sec. 6.4
Variable) on the GPU, against the FP64 oracle electron by electron and
against the closed forms of a constant-frequency gas."""
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


@pytest.fixture(scope="module")
def ctx():
    from paper_1901_08140_gb300 import build as B
    B.build()
    c = bz.Context(0)
    yield c
    c.close()


def _gpu(ctx, gases, check=True, **kw):
    mix = bz.Mixture(ctx, gases)
    sw = bz.run_swarm(ctx, mix, bz.make_config(**kw))
    t = sw.tallies(check=check)
    p = sw.particles()
    sw.close()
    return t, p


def _paired(pg, po):
    same = np.ones(len(po["t"]), bool)
    for k in ["n_real", "n_null", "n_fail", "n_ion", "n_att", "steps", "status"]:
        same &= pg[k] == po[k]
    return same


MODES = {"variable": (bz.BZ_TRIAL_VARIABLE, O.TF_VARIABLE), "binned": (bz.BZ_TRIAL_BINNED, O.TF_BINNED)}


@pytest.mark.parametrize("mode", ["variable", "binned"])
def test_fp64_matches_the_oracle_electron_by_electron(ctx, mode):
    gases = W.ar_co2_mixture()
    kw = dict(e_over_n_Td=30.0, real_collisions=300, seed=41, max_trials=400000)
    strat = dict(zeta=0.4, grace=50, bins_per_decade=8)
    t, p = _gpu(ctx, gases, check=False, n_electrons=2000, precision=64, trial_mode=MODES[mode][0], **kw, **strat)
    m = O.Mixture(gases)
    po = O.run_swarm(m, n=2000, threads=O.cpu_count(), strategy=MODES[mode][1], **kw, **strat)
    assert p["n_fail"].sum() > 0 and po["n_fail"].sum() > 0      # the strategies do fail and revert
    same = _paired(p, po)
    assert same.mean() > 0.99
    # Every decision agrees; values agree to rounding amplified along the
    # trajectory: nu' follows nu(eps), so flight times depend on the energy and
    # the two FP64 rounding orders drift apart, typically to 1e-12 and for a
    # rare electron of a thousand steps to ~1e-6.  The compiled bin maxima
    # carry a 1e-9 guard the oracle's exact maxima do not, which shifts every
    # Binned flight by 1e-9.  A wrong formula would move most electrons, so
    # the median is held at that level and the tail bounded; nu_p is stored
    # in FP32.
    for k in ["z", "t", "sum_e", "nu_p"]:
        # relative to the value, with a floor for coordinates that pass near 0
        scale = np.abs(po[k][same]) + 1e-6 * np.abs(po[k]).mean()
        r = np.abs(p[k][same] - po[k][same]) / scale
        assert np.median(r) < (1e-7 if k == "nu_p" else 1e-8), k
        assert np.quantile(r, 0.99) < (3e-7 if k == "nu_p" else 1e-7) and r.max() < 1e-4, k
    to = OT.swarm_tallies(po, kw["e_over_n_Td"], m.n_total)
    assert t["efficiency"] == pytest.approx(to["efficiency"], rel=1e-3, abs=0.0)


def test_variable_on_a_constant_frequency_gas_fp32(ctx):
    """nu constant: (1 + zeta) nu does not fail, efficiency 1/(1 + zeta), and
    the drift velocity is e E / (m nu).  (Below the table's first point,
    1e-4 eV, nu grows as sqrt(eps): a query there can fail once the electron
    is back above it -- a handful in 1e8 trials.)"""
    from test_oracle_pins import _maxwell_closed_forms
    spec = W.maxwell_swarm(n_electrons=200000, real_collisions=500)
    gas = spec.gases[0]
    t, p = _gpu(ctx, spec.gases, n_electrons=spec.n_electrons, real_collisions=500, e_over_n_Td=spec.e_over_n_Td,
                seed=spec.seed, precision=32, trial_mode=bz.BZ_TRIAL_VARIABLE, zeta=0.25, grace=13)
    trials = t["n_real"] + t["n_null"]
    assert t["n_fail"] < 1e-6 * trials and t["error_flags"] == 0
    se = math.sqrt(0.8 * 0.2 / trials)
    assert abs(t["efficiency"] - 0.8) < 5 * se
    E = spec.e_over_n_Td * 1e-21 * gas.number_density_m3
    vd = QE * E / (ME * 1e12)
    assert abs(t["W"] - vd) < 3.5 * t["W_se"]
    kappa = 2 * ME * gas.mass_kg / (ME + gas.mass_kg) ** 2
    mean_eps, _, _ = _maxwell_closed_forms(500, 0.1, 1e12, kappa, vd)
    assert abs(t["eps"] - mean_eps) < 3.5 * t["eps_se"]


def test_fp32_strategies_agree_with_the_fp64_oracle_statistically(ctx):
    gases = W.ar_co2_mixture()
    kw = dict(e_over_n_Td=60.0, real_collisions=200, seed=43, max_trials=400000)
    for mode in ("variable", "binned"):
        strat = dict(zeta=0.25, grace=100, bins_per_decade=4)
        t, _ = _gpu(ctx, gases, check=False, n_electrons=4000, precision=32, trial_mode=MODES[mode][0], **kw,
                    **strat)
        m = O.Mixture(gases)
        po = O.run_swarm(m, n=4000, threads=O.cpu_count(), strategy=MODES[mode][1], **kw, **strat)
        to = OT.swarm_tallies(po, kw["e_over_n_Td"], m.n_total)
        for k in ["W", "eps", "D_L", "D_T"]:
            se = math.hypot(t[k + "_se"], to[k + "_se"])
            assert abs(t[k] - to[k]) <= 3.5 * se, (mode, k, t[k], to[k], se)


def test_binned_second_fail_is_an_error(ctx):
    """One bin per decade at 300 Td: some electrons fail twice under one
    retry; they stop with ST_TRIAL, the swarm reports BZ_ETRIAL."""
    gases = [W.argon_like()]
    kw = dict(e_over_n_Td=300.0, real_collisions=400, seed=8, max_trials=200000)
    t, p = _gpu(ctx, gases, check=False, n_electrons=400, precision=64, trial_mode=bz.BZ_TRIAL_BINNED,
                bins_per_decade=1, grace=1000, **kw)
    po = O.run_swarm(O.Mixture(gases), n=400, threads=O.cpu_count(), strategy=O.TF_BINNED, bins_per_decade=1,
                     grace=1000, **kw)
    assert t["status"] == bz.BZ_ETRIAL and t["error_flags"] & bz.BZ_ERR_TRIAL
    err = p["status"] == bz.ST_TRIAL
    assert err.any() and np.all(p["n_fail"][err] >= 2)
    assert np.mean(p["status"] == po["status"]) > 0.97


def test_batch_of_adaptive_swarms_equals_alone(ctx):
    specs = W.batched_swarms(count=6, real_collisions=80, max_electrons=20000)
    mixes = [bz.Mixture(ctx, s.gases) for s in specs]
    cfgs = [bz.config_from_spec(s, trial_mode=bz.BZ_TRIAL_VARIABLE if i % 2 else bz.BZ_TRIAL_BINNED,
                                grace=40, max_trials=400000) for i, s in enumerate(specs)]
    alone = []
    for m, c in zip(mixes, cfgs):
        sw = bz.run_swarm(ctx, m, c)
        alone.append(sw.tallies(check=False))
        sw.close()
    b = bz.Batch(ctx, mixes, cfgs)
    b.launch()
    got = b.tallies(check=False)
    b.close()
    for a, g in zip(alone, got):
        for k in ("W", "eps", "D_L", "n_real", "n_null", "n_fail"):
            assert a[k] == g[k] or (a[k] != a[k] and g[k] != g[k]), k


def test_invalid_strategy_configurations(ctx):
    mix = bz.Mixture(ctx, [W.argon_like()])
    bad = [dict(trial_mode=bz.BZ_TRIAL_BINNED, bins_per_decade=3),
           dict(trial_mode=bz.BZ_TRIAL_VARIABLE, zeta=-1.0),
           dict(trial_mode=bz.BZ_TRIAL_VARIABLE, grace=0),
           dict(trial_mode=bz.BZ_TRIAL_VARIABLE, spawn=True, t_end_s=1e-10),
           dict(trial_mode=7)]
    for over in bad:
        with pytest.raises(bz.BzError):
            bz.run_swarm(ctx, mix, bz.make_config(n_electrons=10, real_collisions=10, e_over_n_Td=10.0, **over))
    lazy = bz.make_config(n_electrons=10, real_collisions=10, e_over_n_Td=10.0)
    var = bz.make_config(n_electrons=10, real_collisions=10, e_over_n_Td=10.0, trial_mode=bz.BZ_TRIAL_VARIABLE)
    with pytest.raises(bz.BzError):
        bz.Batch(ctx, [mix, mix], [lazy, var])
