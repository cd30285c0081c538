"""The bounded wait of table staging, made to run out by a failure set up on
the host (hold_stage: a copy that is never issued), on the GPU."""
import time

import pytest

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


def test_stage_wait_gives_up_after_its_limit(ctx):
    """Every block, once its tables are in shared memory, waits on a copy
    that is never issued.  After stage_wait_s it gives up with no copy in
    flight, flags BZ_ERR_STAGE_TIMEOUT and exits: the read reports
    BZ_ETIMEOUT, a batch reports it per swarm, and the context stays usable."""
    mix = bz.Mixture(ctx, W.ar_co2_avalanche_mixture())
    kw = dict(n_electrons=20000, real_collisions=50, e_over_n_Td=100.0, trial_mode=bz.BZ_TRIAL_WINDOW)
    t0 = time.time()
    sw = bz.run_swarm(ctx, mix, bz.make_config(stage_wait_s=0.05, hold_stage=1, **kw))
    with pytest.raises(bz.BzError) as ei:
        sw.tallies()
    elapsed = time.time() - t0
    assert ei.value.status == bz.BZ_ETIMEOUT
    t = sw.tallies(check=False)
    sw.close()
    assert t["error_flags"] & bz.BZ_ERR_STAGE_TIMEOUT
    assert 0.05 <= elapsed < 30.0
    # the batched form: every swarm's read reports the timeout
    cfgs = [bz.make_config(stage_wait_s=0.05, hold_stage=1, seed=W.swarm_seed(i), **kw) for i in range(3)]
    b = bz.Batch(ctx, [mix] * 3, cfgs)
    b.launch()
    with pytest.raises(bz.BzError) as ei:
        b.tallies()
    assert ei.value.status == bz.BZ_ETIMEOUT
    assert all(x["error_flags"] & bz.BZ_ERR_STAGE_TIMEOUT for x in b.tallies(check=False))
    b.close()
    # the context still runs work, with the default wait
    ok = bz.run_swarm(ctx, mix, bz.make_config(**kw))
    t = ok.tallies()
    ok.close()
    assert t["n_real"] == 50 * 20000 and t["error_flags"] == 0

