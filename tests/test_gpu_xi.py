"""xi form of the scattering angle (Eqs. 6-7) on the GPU, against the FP64
oracle electron by electron and statistically."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import tallies as OT
from paper_1901_08140_gb300 import bz
from paper_1901_08140_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1901_08140_gb300 import build as B
    B.build()
    c = bz.Context(0)
    yield c
    c.close()


def _xi_mixture():
    n = W.N_STP_293
    return [W.argon_like(0.9 * n), W.co2_like(0.1 * n, xi_form=True)]


def _gpu(ctx, gases, **kw):
    mix = bz.Mixture(ctx, gases)
    sw = bz.run_swarm(ctx, mix, bz.make_config(**kw))
    t = sw.tallies()
    p = sw.particles()
    sw.close()
    return t, p, mix


def _paired(pg, po):
    same = np.ones(len(po["t"]), bool)
    for k in ["n_real", "n_null", "n_fail", "n_ion", "n_att", "steps", "status"]:
        same &= pg[k] == po[k]
    return same


@pytest.mark.parametrize("mode", [bz.BZ_TRIAL_LAZY, bz.BZ_TRIAL_WINDOW])
def test_fp64_matches_the_oracle(ctx, mode):
    gases = _xi_mixture()
    kw = dict(e_over_n_Td=100.0, real_collisions=300, seed=61)
    t, p, mix = _gpu(ctx, gases, n_electrons=2000, precision=64, trial_mode=mode, **kw)
    assert mix.info["n_xi_gases"] == 1
    po = O.run_swarm(O.Mixture(gases), n=2000, threads=O.cpu_count(), **kw)
    if mode == bz.BZ_TRIAL_WINDOW:
        # the window samples the same process with other draws: statistics only
        to = OT.swarm_tallies(po, kw["e_over_n_Td"], W.N_STP_293)
        for k in ["W", "eps", "D_L", "D_T"]:
            assert abs(t[k] - to[k]) <= 3.5 * math.hypot(t[k + "_se"], to[k + "_se"]), k
        return
    # same draws: electron by electron
    same = _paired(p, po)
    assert same.mean() > 0.99
    for k in ["z", "t", "sum_e"]:
        scale = np.abs(po[k][same]) + 1e-6 * np.abs(po[k]).mean()
        assert np.all(np.abs(p[k][same] - po[k][same]) / scale < 1e-8), k


def test_fp32_statistics_match_the_fp64_oracle(ctx):
    gases = _xi_mixture()
    kw = dict(e_over_n_Td=60.0, real_collisions=300, seed=62)
    t, _, _ = _gpu(ctx, gases, n_electrons=6000, precision=32, **kw)
    po = O.run_swarm(O.Mixture(gases), n=6000, threads=O.cpu_count(), **kw)
    to = OT.swarm_tallies(po, kw["e_over_n_Td"], W.N_STP_293)
    for k in ["W", "eps", "eps_after", "D_L", "D_T"]:
        assert abs(t[k] - to[k]) <= 3.5 * math.hypot(t[k + "_se"], to[k + "_se"]), k


def test_equal_cross_sections_scatter_isotropically(ctx):
    """sigma_el = sigma_mt gives xi = 0, where Eq. 6 is the isotropic law.  The
    isotropic gas draws its new direction in the lab frame and the xi gas
    turns the incident one, so the swarms agree in distribution (every
    statistic within 3.5 combined SE) and first flights agree to rounding."""
    base = W.co2_like()
    grid, s_mt = base.channels[0].energy_eV, base.channels[0].sigma_m2
    iso_xi = W.Gas("xi-iso", base.mass_kg, base.number_density_m3, W.XI_FORM, base.channels, sigma_el=(grid, s_mt))
    kw = dict(n_electrons=20000, e_over_n_Td=40.0, real_collisions=200, seed=63)
    ta, _, _ = _gpu(ctx, [base], **kw)
    tb, _, _ = _gpu(ctx, [iso_xi], **kw)
    for k in ["W", "eps", "eps_after", "D_L", "D_T"]:
        assert abs(ta[k] - tb[k]) <= 3.5 * math.hypot(ta[k + "_se"], tb[k + "_se"]), k
    one = dict(kw, n_electrons=3000, real_collisions=1, precision=64)
    _, a, _ = _gpu(ctx, [base], **one)
    _, b, _ = _gpu(ctx, [iso_xi], **one)
    same = _paired(a, b)   # the two gases run different builds (lean, feature): FP64 rounding may differ
    assert same.mean() > 0.999
    assert np.allclose(a["z"][same], b["z"][same], rtol=1e-12, atol=1e-18)


def test_batches_spawn_and_validation(ctx):
    xi_mix = bz.Mixture(ctx, _xi_mixture())
    plain_mix = bz.Mixture(ctx, [W.argon_like()])
    cfgs = [bz.make_config(n_electrons=3000 + 500 * i, real_collisions=50, e_over_n_Td=30.0 + 20 * i,
                           seed=W.swarm_seed(90 + i)) for i in range(3)]
    alone = []
    for c in cfgs:
        sw = bz.run_swarm(ctx, xi_mix, c)
        alone.append(sw.tallies())
        sw.close()
    b = bz.Batch(ctx, [xi_mix] * 3, cfgs)
    b.launch()
    for a, g in zip(alone, b.tallies()):
        assert a["W"] == g["W"] and a["n_real"] == g["n_real"] and a["n_null"] == g["n_null"]
    b.close()
    # one launch holds one instance of the step kernel
    with pytest.raises(bz.BzError):
        bz.Batch(ctx, [xi_mix, plain_mix], cfgs[:2])
    # an avalanche in the xi mixture runs (spawn mode has every feature)
    sw = bz.run_swarm(ctx, xi_mix, bz.make_config(n_electrons=10, real_collisions=10 ** 9, e_over_n_Td=300.0,
                                                  t_end_s=0.3e-9, spawn=True, pop_cap=10 ** 6, seed=5))
    t = sw.tallies()
    sw.close()
    assert t["n_spawned"] > 0 and t["error_flags"] == 0
