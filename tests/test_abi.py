"""The C ABI library builds, loads and exports every declared symbol; its
host-only logic (configuration, field validation, mixture compilation and
trial frequency) is checked without a GPU."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT
from oracle import oracle as O
from paper_1901_08140_gb300 import build as B
from paper_1901_08140_gb300 import bz
from paper_1901_08140_gb300 import workloads as W


@pytest.fixture(scope="module")
def L():
    B.build()
    return bz.lib()


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(bz_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(bz_\w+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(names) == set(bz.SIGNATURES)
    assert L.bz_abi_version() == 8


def test_struct_layouts_match_the_header(tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "bz.h"\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                    'sizeof(bz_batch_opts),offsetof(bz_batch_opts,block_threads),sizeof(bz_channel),sizeof(bz_gas),sizeof(bz_mixture_opts),sizeof(bz_mixture_info),'
                    'sizeof(bz_swarm_config),sizeof(bz_tallies),sizeof(bz_particles),sizeof(bz_allocator),'
                    'offsetof(bz_tallies,n_particles),offsetof(bz_swarm_config,seed));return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(bz.bz_batch_opts), bz.bz_batch_opts.block_threads.offset, C.sizeof(bz.bz_channel),
            C.sizeof(bz.bz_gas), C.sizeof(bz.bz_mixture_opts), C.sizeof(bz.bz_mixture_info),
            C.sizeof(bz.bz_swarm_config), C.sizeof(bz.bz_tallies), C.sizeof(bz.bz_particles),
            C.sizeof(bz.bz_allocator), bz.bz_tallies.n_particles.offset, bz.bz_swarm_config.seed.offset]
    assert got == want


def test_config_defaults_and_field_validation(L):
    cfg = bz.bz_swarm_config()
    L.bz_config_defaults(C.byref(cfg))
    assert cfg.precision == 32 and cfg.real_collisions == 1000 and cfg.seed == 1901081400
    assert cfg.eps0_mean_eV == 0.1 and cfg.trial_mode == bz.BZ_TRIAL_LAZY
    assert (cfg.zeta, cfg.grace, cfg.bins_per_decade, cfg.gas_temperature_K) == (0.25, 5000, 8, 0.0)
    assert L.bz_set_fields(C.byref(cfg), 10.0, 1.0, 0.5) == bz.BZ_OK
    assert (cfg.e_over_n_Td, cfg.b_T, cfg.b_angle_rad) == (10.0, 1.0, 0.5)
    for bad in [(-1.0, 0.0, 0.0), (float("nan"), 0.0, 0.0), (1.0, -2.0, 0.0), (1.0, 1.0, float("inf"))]:
        assert L.bz_set_fields(C.byref(cfg), *bad) == bz.BZ_EINVAL
        assert bz.bz_last_error()
    assert (cfg.e_over_n_Td, cfg.b_T, cfg.b_angle_rad) == (10.0, 1.0, 0.5)


def test_no_cpu_fallback_without_a_gpu(L):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = L.bz_create(0, None, C.byref(h))
    assert st in (bz.BZ_ECUDA, bz.BZ_EINVAL)
    with pytest.raises(bz.BzError):
        bz.Context(0)


@pytest.mark.parametrize("name", ["maxwell", "argon", "arco2", "batched3"])
def test_host_compiled_trial_frequency_matches_the_oracle(L, name):
    gases = {"maxwell": [W.maxwell_gas()], "argon": [W.argon_like()], "arco2": W.ar_co2_mixture(),
             "batched3": W.batched_swarms(count=4)[3].gases}[name]
    info = bz.compile_info(gases)
    m = O.Mixture(gases)
    assert info["nu_max"] == pytest.approx(m.nu_max, rel=1e-9, abs=0.0)
    assert info["nu_trial"] == pytest.approx(m.nu_max * (1 + 1e-6), rel=1e-9, abs=0.0)
    assert info["n_total"] == pytest.approx(m.n_total, rel=1e-15, abs=0.0)
    n_pts = len(np.unique(np.concatenate([ch.energy_eV for g in gases for ch in g.channels] +
                                         [[ch.threshold_eV] for g in gases for ch in g.channels if ch.kind])))
    assert info["n_records"] == n_pts + 1


def test_host_compiled_trial_frequency_with_inner_tails(L):
    e = np.geomspace(1e-3, 100.0, 300)
    el = W.Channel(W.ELASTIC, 0.0, e, 2e-20 / (1 + e))
    ex = W.Channel(W.EXCITATION, 5.0, np.linspace(5.0, 30.0, 20), np.linspace(0.0, 3e-20, 20))
    gases = [W.Gas("t", 40 * W.ATOMIC_MASS_UNIT, 1e25, W.ISOTROPIC, [el, ex])]
    info = bz.compile_info(gases)
    m = O.Mixture(gases)
    assert info["first_tail_record"] < info["n_records"] - 1
    assert info["nu_max"] == pytest.approx(m.nu_max, rel=1e-9, abs=0.0)
    info2 = bz.compile_info(gases, eps_cap_eV=1000.0)
    m2 = O.Mixture(gases, eps_cap=1000.0)
    assert info2["nu_max"] == pytest.approx(m2.nu_max, rel=1e-9, abs=0.0)


def _bad(kind="ok"):
    e = np.array([1.0, 2.0, 3.0])
    s = np.array([1e-20, 2e-20, 3e-20])
    th, mass, dens, k = 0.0, 1e-26, 1e25, W.ELASTIC
    if kind == "nonmono":
        e = np.array([1.0, 3.0, 2.0])
    elif kind == "neg":
        s = np.array([1e-20, -1e-21, 1e-20])
    elif kind == "nan":
        s = np.array([1e-20, np.nan, 1e-20])
    elif kind == "below_threshold":
        k, th = W.EXCITATION, 2.5
    elif kind == "mass":
        mass = 0.0
    elif kind == "density":
        dens = -1.0
    return [W.Gas("bad", mass, dens, W.ISOTROPIC, [W.Channel(k, th, e, s)])]


def test_xi_form_gases_compile_and_validate():
    n = W.N_STP_293
    info = bz.compile_info([W.argon_like(0.9 * n), W.co2_like(0.1 * n, xi_form=True)])
    assert info["n_xi_gases"] == 1 and info["n_gases"] == 2
    base = W.co2_like()
    no_table = W.Gas("xi", base.mass_kg, base.number_density_m3, W.XI_FORM, base.channels)
    two_elastic = W.Gas("xi", base.mass_kg, base.number_density_m3, W.XI_FORM,
                        base.channels + [base.channels[0]], sigma_el=(base.channels[0].energy_eV,
                                                                     base.channels[0].sigma_m2))
    for gas in (no_table, two_elastic):
        with pytest.raises(bz.BzError):
            bz.compile_info([gas])


@pytest.mark.parametrize("kind", ["nonmono", "neg", "nan", "below_threshold", "mass", "density"])
def test_invalid_tables_are_rejected(L, kind):
    bz.compile_info(_bad("ok"))
    with pytest.raises(bz.BzError) as ei:
        bz.compile_info(_bad(kind))
    assert ei.value.status == bz.BZ_EINVAL
