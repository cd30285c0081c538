"""One swarm run in parts (id ranges, as on several GPUs) merged through its
FP64 tally group sums equals the swarm run whole, on the GPU through the C
ABI: the two-exchange merge (pass-1 sums, the drift they give, pass-2 sums
about it) of separate launches and of swarms in one batch."""
import numpy as np
import pytest

from paper_1901_08140_gb300 import bz
from paper_1901_08140_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("W", "Wx", "Wy", "W_flux", "eps", "eps_after", "alpha", "eta", "D", "D_L", "D_T", "sig", "sig_L", "sig_T",
        "D_L_flux", "D_T_flux", "efficiency", "W_se", "eps_se", "D_L_se", "D_T_se")


@pytest.fixture(scope="module")
def ctx():
    from paper_1901_08140_gb300 import build as B
    B.build()
    c = bz.Context(0)
    yield c
    c.close()


def _check(merged, whole):
    for k in KEYS:
        assert merged[k] == pytest.approx(whole[k], rel=1e-11, abs=1e-300), k
    for k in ("n_particles", "n_real", "n_null", "n_window", "n_ion", "n_att"):
        assert merged[k] == whole[k], k


def test_two_launches_merge_to_one(ctx):
    gases = W.ar_co2_mixture()
    mix = bz.Mixture(ctx, gases)
    kw = dict(real_collisions=200, e_over_n_Td=120.0, b_T=0.7, b_angle_rad=1.0, seed=77,
              trial_mode=bz.BZ_TRIAL_WINDOW)
    n, cut = 30000, 12345
    whole = bz.run_swarm(ctx, mix, bz.make_config(n_electrons=n, **kw))
    tw = whole.tallies()
    a = bz.run_swarm(ctx, mix, bz.make_config(n_electrons=cut, **kw))
    b = bz.run_swarm(ctx, mix, bz.make_config(n_electrons=n - cut, id_offset=cut, **kw))
    g1 = a.group_sums1() + b.group_sums1()
    assert np.allclose(g1, whole.group_sums1(), rtol=1e-12, atol=0)
    d = bz.drift_from_group_sums(g1)
    g2 = a.group_sums2(d) + b.group_sums2(d)
    merged = bz.finalize_group_sums(g1, g2, 120.0, mix.info["n_total"], mix.info["nu_trial"])
    _check(merged, tw)
    for s in (whole, a, b):
        s.close()


def test_swarms_of_a_batch_merge_to_one(ctx):
    mix = bz.Mixture(ctx, [W.argon_like()])
    kw = dict(real_collisions=300, e_over_n_Td=40.0, seed=5, trial_mode=bz.BZ_TRIAL_WINDOW)
    n = 20000
    whole = bz.run_swarm(ctx, mix, bz.make_config(n_electrons=n, **kw))
    tw = whole.tallies()
    whole.close()
    parts = [bz.make_config(n_electrons=7000, **kw), bz.make_config(n_electrons=8000, id_offset=7000, **kw),
             bz.make_config(n_electrons=5000, id_offset=15000, **kw)]
    batch = bz.Batch(ctx, [mix] * 3, parts)
    batch.launch()
    batch.tallies()
    g1 = sum(batch.group_sums1(i) for i in range(3))
    d = bz.drift_from_group_sums(g1)
    g2 = sum(batch.group_sums2(i, d) for i in range(3))
    merged = bz.finalize_group_sums(g1, g2, 40.0, mix.info["n_total"], mix.info["nu_trial"])
    _check(merged, tw)
    # the batch's own tallies are untouched by the second pass about the merged drift
    assert batch.tallies()[0]["n_particles"] == 7000
    batch.close()
