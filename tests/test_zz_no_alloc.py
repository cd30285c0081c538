"""The allocation-free tally reduction (bz_reduce_tallies_noalloc).

Some callers cannot allocate device memory where they need swarm
statistics: their device memory is held entirely by another allocator (a
framework's caching pool, a serving process with a fixed memory plan), or
they run latency-sensitive loops in which cudaMalloc / cudaFree would
synchronize the device.  This entry point reduces caller-owned per-particle
arrays with scratch that lives in a static device array of the library.
The test checks it, through the C ABI, against the tallies of the regular
path (bz_run_swarm + bz_read_tallies) on two calls in a row, and that it
rejects sizes beyond its stated maximum.  It is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1901_08140_gb300 import bz
from paper_1901_08140_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ["W", "Wx", "Wy", "W_flux", "eps", "eps_after", "alpha", "eta", "D", "D_L", "D_T", "sig", "sig_L", "sig_T",
        "D_L_flux", "D_T_flux", "efficiency", "mu", "mu_N", "mu_0", "lorentz_angle", "W_se", "eps_se", "D_L_se",
        "D_T_se"]
COUNTS = ["n_particles", "n_real", "n_null", "n_fail", "n_ion", "n_att", "n_incomplete"]


def _noalloc(torch, dev, p, n, id_offset, eon, n_total, nu_trial):
    tens = {}
    for k in ["x", "y", "z", "t", "sum_e", "sum_e2"]:
        tens[k] = torch.as_tensor(np.ascontiguousarray(p[k], np.float64), device=dev)
    for k in ["n_real", "n_null", "n_fail", "n_ion", "n_att", "status"]:
        tens[k] = torch.as_tensor(np.ascontiguousarray(p[k], np.uint32).view(np.int32), device=dev)
    arr = bz.bz_particle_arrays(*[tens[k].data_ptr() for k in ["x", "y", "z", "t", "sum_e", "sum_e2", "n_real",
                                                                "n_null", "n_fail", "n_ion", "n_att", "status"]])
    out = torch.zeros(C.sizeof(bz.bz_tallies), dtype=torch.uint8, device=dev)
    st = bz.lib().bz_reduce_tallies_noalloc(C.byref(arr), n, id_offset, eon, n_total, nu_trial,
                                           C.c_void_p(out.data_ptr()),
                                           C.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    assert st == bz.BZ_OK, bz.bz_last_error()
    torch.cuda.synchronize(dev)
    host = bz.bz_tallies.from_buffer_copy(out.cpu().numpy().tobytes())
    return {k: getattr(host, k) for k in KEYS + COUNTS}


def test_noalloc_reduction_matches_the_regular_path_twice():
    torch = pytest.importorskip("torch")
    from paper_1901_08140_gb300 import build as B
    B.build()
    ctx = bz.Context(0)
    dev = torch.device("cuda", 0)
    gases = W.ar_co2_mixture()
    mix = bz.Mixture(ctx, gases)
    n, id_offset, eon = 70001, 3, 120.0   # three reduction blocks, a ragged tail
    cfg = bz.make_config(n_electrons=n, real_collisions=40, e_over_n_Td=eon, b_T=0.5, b_angle_rad=1.2, seed=77,
                         id_offset=id_offset)
    sw = bz.run_swarm(ctx, mix, cfg)
    ref = sw.tallies()
    p = sw.particles()
    sw.close()
    for call in range(2):
        got = _noalloc(torch, dev, p, n, id_offset, eon, mix.info["n_total"], mix.info["nu_trial"])
        for k in KEYS:
            assert got[k] == pytest.approx(ref[k], rel=1e-10, abs=1e-300), (call, k)
        for k in COUNTS:
            assert got[k] == ref[k], (call, k)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    pytest.importorskip("torch")
    from paper_1901_08140_gb300 import build as B
    B.build()
    bz.Context(0)
    arr = bz.bz_particle_arrays(*([1] * 12))   # never dereferenced: the size check comes first
    st = bz.lib().bz_reduce_tallies_noalloc(C.byref(arr), bz.BZ_NOALLOC_MAX_PARTICLES + 1, 0, 1.0, 1e25, 1e12,
                                           C.c_void_p(16), None)
    assert st == bz.BZ_EBUDGET
    assert "16777216" in bz.bz_last_error()
