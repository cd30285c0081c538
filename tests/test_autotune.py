"""Autotuner: workload signature, cache round trip, and (GPU) a tuned batch."""
import pytest

from paper_1901_08140_gb300 import autotune, bz
from paper_1901_08140_gb300 import build as B
from paper_1901_08140_gb300 import workloads as W


@pytest.fixture(scope="module")
def L():
    B.build()
    return bz.lib()


def test_signature_and_apply(L):
    cfgs = [bz.make_config(n_electrons=1000 * (i + 1), real_collisions=100, e_over_n_Td=10.0,
                           trial_mode=bz.BZ_TRIAL_WINDOW if i % 2 else bz.BZ_TRIAL_LAZY) for i in range(4)]
    sig = autotune.signature(cfgs)
    assert sig == "n4-e13-m0.2-p32"
    out = autotune.apply(cfgs, {"window_c": 3.0, "tiles_per_block": 16, "blocks_per_sm": 0})
    assert [c.window_c for c in out] == [0.0, 3.0, 0.0, 3.0]
    assert [c.window_c for c in cfgs] == [0.0, 0.0, 0.0, 0.0]   # inputs untouched


def test_cache_round_trip(tmp_path, L):
    path = str(tmp_path / "cache.json")
    assert autotune.load_cache(path) == {}
    autotune.store_cache({"gpu|sig": {"window_c": 1.5, "tiles_per_block": 8, "blocks_per_sm": 2}}, path)
    assert autotune.load_cache(path)["gpu|sig"]["tiles_per_block"] == 8


def test_tile_size_from_tiles_per_block(L):
    cfgs = [bz.make_config(n_electrons=n, real_collisions=10, e_over_n_Td=1.0) for n in (10 ** 6, 3 * 10 ** 5)]
    # 1.3e6 electrons over 152 SMs x 3 blocks x 16 tiles: 179 -> 256 (the floor); x 1 tile: 2851 -> 3072
    assert autotune.tile_size(cfgs, {"tiles_per_block": 16, "blocks_per_sm": 0}) == 256
    assert autotune.tile_size(cfgs, {"tiles_per_block": 1, "blocks_per_sm": 0}) == 3072
    assert autotune.tile_size(cfgs, {"tiles_per_block": 1, "blocks_per_sm": 2}) == 4352
    # blocks of 128 threads: 6 resident per SM, tiles of half the electrons (1426 -> 1536); 384: 2 per SM
    assert autotune.tile_size(cfgs, {"tiles_per_block": 1, "blocks_per_sm": 0, "block_threads": 128}) == 1536
    assert autotune.tile_size(cfgs, {"tiles_per_block": 1, "blocks_per_sm": 0, "block_threads": 384}) == 4352


def test_cached_choice_and_the_table_budget(tmp_path, L):
    """A cached choice is returned as it is to a caller that passed the gas
    lists; a caller without them gets the library's table budget (it runs
    on the mixtures it compiled)."""
    cfgs = [bz.make_config(n_electrons=5000, real_collisions=10, e_over_n_Td=1.0) for _ in range(3)]
    path = str(tmp_path / "cache.json")
    choice = dict(autotune.DEFAULT, block_threads=768, smem_budget=autotune.ONE_BLOCK_BUDGET)
    autotune.store_cache({"GPU|" + autotune.signature(cfgs): choice}, path)
    with_gases = autotune.tune(None, [], cfgs, cache_path=path, gpu_name="GPU", gas_lists=[[], [], []])
    assert with_gases["cached"] is True and with_gases["smem_budget"] == autotune.ONE_BLOCK_BUDGET
    without = autotune.tune(None, [], cfgs, cache_path=path, gpu_name="GPU")
    assert without["block_threads"] == 768 and without["smem_budget"] == 0


@pytest.mark.gpu
def test_tune_a_small_batch(tmp_path, L):
    ctx = bz.Context(0)
    specs = W.argon_sweep(n_electrons=20000, real_collisions=200, points=4)
    mix = bz.Mixture(ctx, specs[0].gases)
    cfgs = [bz.config_from_spec(s, trial_mode=bz.BZ_TRIAL_WINDOW) for s in specs]
    path = str(tmp_path / "c.json")
    choice = autotune.tune(ctx, [mix] * 4, cfgs, cache_path=path)
    assert choice["cached"] is False and choice["window_c"] in autotune.WINDOW_C
    assert mix.info["channels_in_smem"] == 1 and choice["channels_in_l2"] in (False, True)
    assert choice["block_threads"] in autotune.BLOCK_THREADS
    again = autotune.tune(ctx, [mix] * 4, cfgs, cache_path=path)
    assert again["cached"] is True and again["window_c"] == choice["window_c"]
    b = autotune.make_batch(ctx, [mix] * 4, autotune.apply(cfgs, choice), choice)
    b.launch()
    assert all(t["n_real"] == 20000 * 200 and t["error_flags"] == 0 for t in b.tallies())
    b.close()
