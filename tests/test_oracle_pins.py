"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a closed form, an exact invariant, a
brute-force computation or a value printed in the paper, chosen so that a
plausible slip (dropped term, wrong sign, swapped operand, wrong index) in
the corresponding oracle function fails.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

from conftest import read_golden
from oracle import oracle as O
from oracle import tallies as T
from paper_1901_08140_gb300 import workloads as W

QE = 1.602176634e-19
ME = 9.1093837015e-31
HARTREE = 27.211386245988


# --------------------------------------------------------------------------
# Random numbers: the method asks for independent uniforms on [0,1)
# (Eqs. 3, 4, 5); these pins check exactly that.
# --------------------------------------------------------------------------
def _words(n, step=0, sub=0, key=(12345, 678)):
    return np.array([O.philox([i, 0, step, sub], key) for i in range(n)], dtype=np.uint64)


def test_philox_uniformity_and_independence():
    w = _words(20000)
    u = (((w >> 9).astype(np.float64)) + 0.5) / 2 ** 23
    flat = u.ravel()
    assert abs(flat.mean() - 0.5) < 4 * math.sqrt(1 / 12 / flat.size)
    assert abs(flat.var() - 1 / 12) < 0.01 * (1 / 12)
    counts, _ = np.histogram(flat, bins=64, range=(0, 1))
    assert stats.chisquare(counts).pvalue > 1e-4
    # the four words of one call and consecutive counters are uncorrelated
    for a, b in [(0, 1), (1, 2), (2, 3), (0, 3)]:
        r = np.corrcoef(u[:, a], u[:, b])[0, 1]
        assert abs(r) < 4 / math.sqrt(len(u))
    r = np.corrcoef(u[:-1, 0], u[1:, 0])[0, 1]
    assert abs(r) < 4 / math.sqrt(len(u))
    # every 32-bit output bit is balanced
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint64)) & 1).reshape(-1, 32).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / math.sqrt(w.size))


def _curand_host_philox(seed: int, n_blocks: int) -> np.ndarray:
    """The first n_blocks x 4 words of cuRAND's host-side Philox4_32_10
    generator seeded with `seed` (NVIDIA's implementation of the same
    published generator), or None where libcurand is not installed."""
    import ctypes
    import ctypes.util
    paths = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so"),
             ctypes.util.find_library("curand")]
    lib = None
    for p in paths:
        try:
            lib = ctypes.CDLL(p) if p else None
        except OSError:
            lib = None
        if lib is not None:
            break
    if lib is None:
        return None
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4 * n_blocks, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(-1, 4)


def test_philox_identity_against_curand():
    """Known answers of Philox4x32-10 (Salmon et al. 2011) from an
    implementation that is not this project's: cuRAND's host generator.
    Seeded with s, its block k is Philox at counter (k div 65536, 0, k mod
    65536, 0) under the key (s mod 2^32, s div 2^32).  Over two sweeps of
    the third counter word and three keys this fixes the multipliers, the
    Weyl constants of the key schedule, the word permutation of a round and
    the number of rounds: swapping two multipliers or two high words, or a
    wrong Weyl constant, changes every block."""
    n = 2 * 65536 + 8
    for seed in (0, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF):
        ref = _curand_host_philox(seed, n)
        if ref is None:
            pytest.skip("libcurand is not installed")
        key = [seed & 0xFFFFFFFF, seed >> 32]
        rng = np.random.default_rng(seed & 0xFFFF)
        ks = np.concatenate([np.arange(0, 64), np.arange(65530, 65542), np.arange(131068, n),
                             rng.integers(0, n, 400)])
        for k in ks:
            k = int(k)
            got = O.philox([k // 65536, 0, k % 65536, 0], key)
            assert np.array_equal(got, ref[k]), (seed, k, got, ref[k])


def test_philox_counter_and_key_avalanche():
    base = O.philox([7, 0, 3, 0], [1, 2]).astype(np.uint64)
    flips = []
    for word in range(4):
        for bit in (0, 13, 31):
            ctr = [7, 0, 3, 0]
            ctr[word] ^= 1 << bit
            o = O.philox(ctr, [1, 2]).astype(np.uint64)
            flips.append(sum(bin(int(a ^ b)).count("1") for a, b in zip(base, o)))
    for kw in range(2):
        key = [1, 2]
        key[kw] ^= 1 << 5
        o = O.philox([7, 0, 3, 0], key).astype(np.uint64)
        flips.append(sum(bin(int(a ^ b)).count("1") for a, b in zip(base, o)))
    assert 56 < np.mean(flips) < 72  # 128 bits, half flip on average


def test_uniform_open_interval_lattice():
    assert O.uniform(0) == 0.5 / 2 ** 23
    assert O.uniform(0xFFFFFFFF) == 1 - 0.5 / 2 ** 23
    assert O.uniform(0x1FF) == O.uniform(0)         # only the top 23 bits count
    assert O.uniform(1 << 9) == 1.5 / 2 ** 23
    # every value is exactly representable in FP32
    for w in (0, 1 << 9, 0x80000000, 0xFFFFFFFF, 0x12345678, 0xDEADBEEF):
        u = O.uniform(w)
        assert float(np.float32(u)) == u


# --------------------------------------------------------------------------
# Tables and their extension (Sec. 2.2, Eqs. 12-14), worked by hand.
# --------------------------------------------------------------------------
def _gas(channels, mass=40 * W.ATOMIC_MASS_UNIT, n=1e25, angular=W.ISOTROPIC):
    return W.Gas("t", mass, n, angular, channels)


def test_table_interpolation_and_extension_by_hand():
    el = W.Channel(W.ELASTIC, 0.0, np.array([1.0, 10.0]), np.array([1e-20, 1e-21]))
    ex = W.Channel(W.EXCITATION, 2.0, np.array([3.0, 5.0]), np.array([4e-21, 6e-21]))
    at = W.Channel(W.ATTACHMENT, 3.0, np.array([3.0, 4.0, 6.0]), np.array([0.0, 2e-22, 0.0]))
    m = O.Mixture([_gas([el, ex, at])])
    # elastic: constant to the left, linear inside, power law to the right
    assert m.sigma(0, 0.01) == 1e-20
    assert m.sigma(0, 5.5) == pytest.approx(1e-20 + (1e-21 - 1e-20) * 4.5 / 9.0, rel=1e-14, abs=0.0)
    # K = ln(0.1)/ln(10) = -1, A = 1e-21 * 10: sigma(100) = 1e-22, sigma(20) = 5e-22
    assert m.sigma(0, 100.0) == pytest.approx(1e-22, rel=1e-12, abs=0.0)
    assert m.sigma(0, 20.0) == pytest.approx(5e-22, rel=1e-12, abs=0.0)
    # inelastic: zero below threshold, linear rise from (threshold, 0) to the first point
    assert m.sigma(1, 1.99) == 0.0
    assert m.sigma(1, 2.5) == pytest.approx(2e-21, rel=1e-14, abs=0.0)
    assert m.sigma(1, 4.0) == pytest.approx(5e-21, rel=1e-14, abs=0.0)
    # K = ln(6/4)/ln(5/3); sigma(15) = 6e-21 * 3^K
    K = math.log(1.5) / math.log(5 / 3)
    assert m.sigma(1, 15.0) == pytest.approx(6e-21 * 3 ** K, rel=1e-12, abs=0.0)
    # a table ending in zero extends with zero
    assert m.sigma(2, 5.0) == pytest.approx(1e-22, rel=1e-14, abs=0.0)
    assert m.sigma(2, 50.0) == 0.0
    # Eq. (2): nu = sqrt(2 eps/m) sum n sigma
    eps = 4.0
    S = 1e25 * (m.sigma(0, eps) + m.sigma(1, eps) + m.sigma(2, eps))
    assert m.nu(eps) == pytest.approx(math.sqrt(2 * eps * QE / ME) * S, rel=1e-14, abs=0.0)


def test_density_weighting_of_components():
    el1 = W.Channel(W.ELASTIC, 0.0, np.array([1.0, 10.0]), np.array([1e-20, 1e-20]))
    el2 = W.Channel(W.ELASTIC, 0.0, np.array([1.0, 10.0]), np.array([3e-20, 3e-20]))
    m = O.Mixture([_gas([el1], n=2e25), _gas([el2], n=1e25)])
    eps = 2.0
    assert m.nu(eps) == pytest.approx(math.sqrt(2 * eps * QE / ME) * (2e25 * 1e-20 + 1e25 * 3e-20), rel=1e-14, abs=0.0)


# --------------------------------------------------------------------------
# Trial frequency: exact maximum of nu over [0, eps_cap] (Sec. 6.2).
# --------------------------------------------------------------------------
def _inner_tail_gas():
    e = np.geomspace(1e-3, 100.0, 300)
    el = W.Channel(W.ELASTIC, 0.0, e, 2e-20 / (1 + e))
    ex = W.Channel(W.EXCITATION, 5.0, np.linspace(5.0, 30.0, 20), np.linspace(0.0, 3e-20, 20))
    return _gas([el, ex])


@pytest.mark.parametrize("name", ["maxwell", "argon", "arco2", "inner_tail"])
def test_majorant_matches_brute_force(name):
    gases = {"maxwell": [W.maxwell_gas()], "argon": [W.argon_like()], "arco2": W.ar_co2_mixture(),
             "inner_tail": [_inner_tail_gas()]}[name]
    m = O.Mixture(gases)
    cap = max(float(ch.energy_eV[-1]) for g in gases for ch in g.channels)
    pts = [np.geomspace(1e-7, cap, 400000), np.linspace(0.0, cap, 400000)]
    for g in gases:
        for ch in g.channels:
            pts.append(ch.energy_eV[ch.energy_eV <= cap])
    grid = np.unique(np.concatenate(pts))
    brute = m.nu_many(grid).max()
    assert brute <= m.nu_max * (1 + 1e-12)
    assert brute >= m.nu_max * (1 - 1e-6)


# --------------------------------------------------------------------------
# Channel choice and null fraction (Eqs. 2 and 4): chi-square against the
# table ratios, through the whole trial step with no field.
# --------------------------------------------------------------------------
def test_channel_frequencies_match_table_ratios():
    gas = W.argon_like()
    m = O.Mixture([gas])
    eps = 14.0
    speed = math.sqrt(2 * eps * QE / ME)
    n = 200000
    state = np.zeros((n, 8))
    state[:, 5] = speed
    state[:, 7] = m.nu_max
    ids = np.arange(n, dtype=np.uint64)
    out, dec, eps_io = O.step_replay(m, state, ids, np.full(n, 5, np.uint32), e_over_n_Td=0.0, seed=99)
    assert np.allclose(eps_io[:, 0], eps, rtol=1e-12)
    nu_ch = np.array([gas.number_density_m3 * m.sigma(c, eps) * speed for c in range(m.n_channels)])
    p = np.concatenate([[1 - nu_ch.sum() / m.nu_max], nu_ch / m.nu_max])
    assert p[-1] == 0.0  # ionization is closed at 14 eV
    keep = p > 0
    counts = np.array([np.sum(dec == O.DEC_NULL)] + [np.sum(dec == c) for c in range(m.n_channels)])
    assert counts[~keep].sum() == 0
    assert stats.chisquare(counts[keep], p[keep] * n).pvalue > 1e-4


# --------------------------------------------------------------------------
# Scattering angle (Eq. 5) and energy exchange (Eqs. 8, 9).
# --------------------------------------------------------------------------
def test_isotropic_angle_moments():
    R = (np.arange(100000) + 0.5) / 100000
    c = np.array([O.cos_theta(W.ISOTROPIC, 3.0, r) for r in R])
    assert abs(c.mean()) < 1e-9
    assert c.var() == pytest.approx(1 / 3, rel=1e-6, abs=0.0)


@pytest.mark.parametrize("eps", [0.0, 0.01, 1.0, 27.0, 300.0])
def test_screened_coulomb_mean_deflection(eps):
    R = (np.arange(200000) + 0.5) / 200000
    c = np.array([O.cos_theta(W.SCREENED_COULOMB, eps, r) for r in R])
    cc = 8 * eps / HARTREE
    exact = 1.0 if cc == 0 else (2 / cc ** 2) * ((1 + cc) * math.log1p(cc) - cc)
    assert np.mean(1 - c) == pytest.approx(exact, rel=1e-6, abs=0.0)
    assert np.all(c <= 1) and np.all(c >= -1)


def _two_body(m, M, eps_i, eps_k, cos_cm, rng):
    """Electron (mass m) on a target at rest, exact kinematics in the CM frame."""
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    v = math.sqrt(2 * eps_i * QE / m) * d
    V = m * v / (m + M)
    u = v - V                                # electron in the CM frame
    mu = m * M / (m + M)
    E_cm = 0.5 * mu * (v @ v)                # kinetic energy available in the CM frame
    scale = math.sqrt(1 - eps_k * QE / E_cm)
    a = np.cross(d, [1.0, 0.0, 0.0] if abs(d[0]) < 0.9 else [0.0, 1.0, 0.0])
    a /= np.linalg.norm(a)
    sin_cm = math.sqrt(1 - cos_cm ** 2)
    u_new = scale * np.linalg.norm(u) * (cos_cm * d + sin_cm * a)
    v_new = V + u_new
    U_new = V - (m / M) * u_new              # target, from momentum conservation
    # conservation checks of the construction itself
    assert np.allclose(m * v, m * v_new + M * U_new, rtol=1e-12, atol=1e-40)
    ke0 = 0.5 * m * (v @ v)
    ke1 = 0.5 * m * (v_new @ v_new) + 0.5 * M * (U_new @ U_new) + eps_k * QE
    assert ke1 == pytest.approx(ke0, rel=1e-12, abs=0.0)
    return 0.5 * m * (v_new @ v_new) / QE / eps_i


def test_energy_exchange_matches_two_body_kinematics():
    rng = np.random.default_rng(3)
    for _ in range(300):
        M = rng.uniform(1.0, 200.0) * W.ATOMIC_MASS_UNIT
        if rng.uniform() < 0.3:
            M = rng.uniform(2.0, 50.0) * ME       # light targets exercise the mass terms
        eps_i = float(np.exp(rng.uniform(-2, 5)))
        cos_cm = rng.uniform(-1, 1)
        assert O.ratio_elastic(ME, M, cos_cm) == pytest.approx(_two_body(ME, M, eps_i, 0.0, cos_cm, rng), rel=1e-11, abs=0.0)
        eps_k = eps_i * rng.uniform(0.0, 0.95) * M / (ME + M)
        got = O.ratio_inelastic(ME, M, eps_i, eps_k, cos_cm)
        assert got == pytest.approx(_two_body(ME, M, eps_i, eps_k, cos_cm, rng), rel=1e-10, abs=1e-13)


def test_mean_elastic_loss_is_kappa():
    M = 40 * W.ATOMIC_MASS_UNIT
    kappa = 2 * ME * M / (ME + M) ** 2
    R = (np.arange(50000) + 0.5) / 50000
    r = np.array([O.ratio_elastic(ME, M, O.cos_theta(W.ISOTROPIC, 1.0, x)) for x in R])
    assert np.mean(1 - r) == pytest.approx(kappa, rel=1e-8, abs=0.0)


def test_inelastic_closed_band_is_clamped():
    M = 40 * W.ATOMIC_MASS_UNIT
    assert O.ratio_inelastic(ME, M, 11.5, 11.5, 1.0) == 0.0
    assert O.ratio_inelastic(ME, M, 11.5 * (1 + 0.5 * ME / M), 11.5, -1.0) == 0.0


def test_rotation_geometry():
    rng = np.random.default_rng(5)
    for _ in range(500):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        ct = rng.uniform(-1, 1)
        phi = rng.uniform(0, 2 * math.pi)
        o = O.rotate(d, ct, phi)
        assert np.linalg.norm(o) == pytest.approx(1.0, abs=1e-14)
        assert o @ d == pytest.approx(ct, abs=1e-14)
    # uniform azimuth averages to the axis
    d = np.array([0.3, -0.5, 0.8])
    d /= np.linalg.norm(d)
    phis = (np.arange(720) + 0.5) * 2 * math.pi / 720
    mean = np.mean([O.rotate(d, 0.2, p) for p in phis], axis=0)
    assert np.allclose(mean, 0.2 * d, atol=1e-12)
    # a quarter turn of azimuth gives an orthogonal transverse part
    t0 = O.rotate(d, 0.0, 0.0)
    t1 = O.rotate(d, 0.0, math.pi / 2)
    assert abs(t0 @ t1) < 1e-14 and abs(t0 @ d) < 1e-14


# --------------------------------------------------------------------------
# Motion in uniform static E and B (Sec. 3.6): closed form against RK4.
# --------------------------------------------------------------------------
def _rk4(x, v, accel_E, qm, Bv, T, steps):
    dt = T / steps

    def f(v):
        return accel_E + qm * np.cross(v, Bv)

    for _ in range(steps):
        k1v = f(v); k1x = v
        k2v = f(v + 0.5 * dt[:, None] * k1v); k2x = v + 0.5 * dt[:, None] * k1v
        k3v = f(v + 0.5 * dt[:, None] * k2v); k3x = v + 0.5 * dt[:, None] * k2v
        k4v = f(v + dt[:, None] * k3v); k4x = v + dt[:, None] * k3v
        x = x + dt[:, None] / 6 * (k1x + 2 * k2x + 2 * k3x + k4x)
        v = v + dt[:, None] / 6 * (k1v + 2 * k2v + 2 * k3v + k4v)
    return x, v


@pytest.mark.parametrize("b_T,angle", [(0.1, 0.0), (1.0, math.pi / 2), (2.0, math.pi / 6), (0.7, 2.4)])
def test_motion_matches_rk4(b_T, angle):
    rng = np.random.default_rng(11)
    n_total, eon = W.N_STP_293, 100.0
    E = eon * 1e-21 * n_total
    omega = QE * b_T / ME
    n = 40
    x0 = rng.normal(size=(n, 3)) * 1e-5
    v0 = rng.normal(size=(n, 3)) * 1e6
    T = rng.uniform(0.01, 10.0, size=n) / omega
    # the electron (q = -e) is pushed along +z: E points along -z
    accel = np.array([0.0, 0.0, QE * E / ME])
    Bv = b_T * np.array([math.sin(angle), 0.0, math.cos(angle)])
    xr, vr = _rk4(x0.copy(), v0.copy(), accel, -QE / ME, Bv, T, 6000)
    for i in range(n):
        xo, vo = O.move(x0[i], v0[i], T[i], eon, n_total, b_T, angle)
        scale_x = np.linalg.norm(v0[i]) * T[i] + 1e-3 * np.linalg.norm(x0[i])
        assert np.allclose(xo, xr[i], rtol=0, atol=1e-9 * scale_x + 1e-12 * np.linalg.norm(x0[i]))
        assert np.allclose(vo, vr[i], rtol=0, atol=1e-9 * (np.linalg.norm(v0[i]) + E / b_T))
        # B does no work: the kinetic energy change equals the work of the electric force
        dke = 0.5 * ME * (vo @ vo - v0[i] @ v0[i])
        assert dke == pytest.approx(QE * E * (xo[2] - x0[i][2]), rel=1e-8, abs=1e-12 * 0.5 * ME * (v0[i] @ v0[i]))


def test_motion_without_b_is_a_parabola_and_guiding_centre_drifts_at_exb():
    E = 10.0 * 1e-21 * W.N_STP_293
    a = QE * E / ME
    x, v = O.move([1.0, 2.0, 3.0], [4.0, 5.0, 6.0], 1e-9, 10.0, W.N_STP_293)
    assert np.allclose(x, [1 + 4e-9, 2 + 5e-9, 3 + 6e-9 + 0.5 * a * 1e-18], rtol=1e-15)
    assert np.allclose(v, [4.0, 5.0, 6.0 + a * 1e-9], rtol=1e-15)
    # B along x, E along -z: E x B / B^2 = (-E z) x (B x) / B^2 = -(E/B) y
    b = 1.0
    omega = QE * b / ME
    periods = 1000.0
    T = periods * 2 * math.pi / omega
    x, v = O.move([0.0, 0.0, 0.0], [3e5, -2e5, 1e5], T, 100.0, W.N_STP_293, b, math.pi / 2)
    E100 = 100.0 * 1e-21 * W.N_STP_293
    assert x[1] / T == pytest.approx(-E100 / b, rel=1e-6, abs=0.0)
    assert abs(x[2]) < 1e-4 * abs(x[1])
    assert x[0] == pytest.approx(3e5 * T, rel=1e-9, abs=0.0)  # motion along B is free


# --------------------------------------------------------------------------
# Whole step loop: the constant-frequency Maxwell model has closed forms.
# --------------------------------------------------------------------------
def _maxwell_closed_forms(I, eps0, nu, kappa, vd):
    mvd2 = ME * vd * vd / QE                   # eV
    B = np.empty(I)
    B[0] = eps0 + mvd2
    for i in range(1, I):
        B[i] = (1 - kappa) * B[i - 1] + mvd2
    mean_eps = B.mean()
    # E[v_x^2] of flight i (0 = initial flight), in (m/s)^2
    vx2 = np.empty(I)
    vx2[0] = 2 * eps0 * QE / (3 * ME)
    vx2[1:] = 2 * QE / (3 * ME) * (1 - kappa) * B[:-1]
    DT = vx2.sum() / (nu * I)
    DL = (vx2.sum() + I * vd * vd) / (nu * I)
    return mean_eps, DT, DL


def _group_se(vals_per_group):
    v = np.asarray(vals_per_group)
    return np.std(v, ddof=1) / math.sqrt(len(v))


def test_maxwell_model_closed_forms():
    spec = W.maxwell_swarm(n_electrons=10000, real_collisions=1000)
    gas = spec.gases[0]
    m = O.Mixture(spec.gases)
    p = O.run_swarm(m, e_over_n_Td=spec.e_over_n_Td, real_collisions=spec.real_collisions,
                    n=spec.n_electrons, seed=spec.seed, eps0_mean_eV=spec.eps0_mean_eV,
                    threads=O.cpu_count())
    assert np.all(p["n_real"] == 1000) and np.all(p["n_fail"] == 0)
    nu = 1e12
    E = spec.e_over_n_Td * 1e-21 * gas.number_density_m3
    vd = QE * E / (ME * nu)
    assert vd == pytest.approx(4.40316e4, rel=1e-5, abs=0.0)
    M = gas.mass_kg
    kappa = 2 * ME * M / (ME + M) ** 2
    mean_eps, DT, DL = _maxwell_closed_forms(1000, 0.1, nu, kappa, vd)
    assert mean_eps == pytest.approx(5.2580, abs=5e-4)
    assert DT == pytest.approx(0.61523, rel=1e-4, abs=0.0)
    assert DL == pytest.approx(0.61717, rel=1e-4, abs=0.0)
    tr = T.swarm_tallies(p, spec.e_over_n_Td, gas.number_density_m3)
    assert abs(tr["W"] - vd) < 3 * tr["W_se"]
    assert abs(tr["eps"] - mean_eps) < 3 * tr["eps_se"]
    assert tr["eps_after"] == pytest.approx((1 - kappa) * tr["eps"], rel=2e-4, abs=0.0)
    g = p["id"] % 32
    x, y, z, t = p["x"], p["y"], p["z"], p["t"]
    est_T = [np.sum(x[g == j] ** 2 + y[g == j] ** 2) / (4 * np.sum(t[g == j])) for j in range(32)]
    est_L = [np.sum((z[g == j] - vd * t[g == j]) ** 2) / (2 * np.sum(t[g == j])) for j in range(32)]
    est_W = [np.sum(z[g == j]) / np.sum(t[g == j]) for j in range(32)]
    assert abs(np.sum(x ** 2 + y ** 2) / (4 * np.sum(t)) - DT) < 3 * _group_se(est_T)
    assert abs(np.sum((z - vd * t) ** 2) / (2 * np.sum(t)) - DL) < 3 * _group_se(est_L)
    assert abs(np.sum(z) / np.sum(t) - vd) < 3 * _group_se(est_W)
    # the mean flight time is 1/nu
    assert np.mean(t) == pytest.approx(1000 / nu, rel=3 * math.sqrt(1000) / 1000 / math.sqrt(10000) * 3, abs=0.0)


def test_initial_velocities_are_maxwellian_with_mean_energy():
    v = O.initial_velocities(0.1, 77, 0, 200000)
    eps = 0.5 * ME * np.sum(v * v, axis=1) / QE
    assert abs(eps.mean() - 0.1) < 4 * eps.std() / math.sqrt(len(eps))
    sv = math.sqrt((2 / 3) * 0.1 * QE / ME)
    for k in range(3):
        assert stats.kstest(v[:, k] / sv, "norm").pvalue > 1e-4


# --------------------------------------------------------------------------
# Collision bookkeeping: ionization split and dummy attachment (readings).
# --------------------------------------------------------------------------
def test_ionization_split_and_attachment_energy_accounting():
    gases = [W.co2_like()]
    m = O.Mixture(gases)
    rng = np.random.default_rng(9)
    n = 60000
    eps = np.where(rng.uniform(size=n) < 0.5, 40.0, 4.4)
    speed = np.sqrt(2 * eps * QE / ME)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    state = np.zeros((n, 8))
    state[:, 3:6] = d * speed[:, None]
    state[:, 7] = np.array([m.nu(e) for e in eps]) * (1 + 1e-9)   # nearly every trial is real
    ids = np.arange(n, dtype=np.uint64)
    steps = np.full(n, 3, np.uint32)
    seed = 4242
    out, dec, eio = O.step_replay(m, state, ids, steps, e_over_n_Td=0.0, seed=seed)
    kinds = m.ch_kind
    ion = np.array([c >= 0 and kinds[c] == W.IONIZATION for c in dec])
    att = np.array([c >= 0 and kinds[c] == W.ATTACHMENT for c in dec])
    assert ion.sum() > 20 and att.sum() > 3
    for i in np.nonzero(ion)[0]:
        c = dec[i]
        u = [O.uniform(w) for w in O.philox([i, 0, 3, 0], [seed, 0])]
        w4 = O.uniform(O.philox([i, 0, 3, 1], [seed, 0])[0])
        M = m.gas_mass[m.ch_gas[c]]
        # isotropic gas: the new direction is drawn in the lab frame (polar cosine
        # 1 - 2 u2, azimuth 2 pi u3) and Eq. 9 takes its cosine to the incident one
        cl = 1 - 2 * u[2]
        sl = math.sqrt(max(0.0, 1 - cl * cl))
        ct = float(d[i] @ np.array([sl * math.cos(2 * math.pi * u[3]), sl * math.sin(2 * math.pi * u[3]), cl]))
        r = O.ratio_inelastic(ME, M, eps[i], m.ch_threshold[c], ct)
        assert eio[i, 1] == pytest.approx(r * (1 - w4) * eps[i], rel=1e-12, abs=0.0)
        ef = 0.5 * ME * np.sum(out[i, 3:6] ** 2) / QE
        assert ef == pytest.approx(eio[i, 1], rel=1e-10, abs=0.0)
    assert np.all(eio[att, 1] == 0.0) and np.all(out[att, 3:6] == 0.0)


def test_ionization_energy_moments_match_eq9_closed_forms():
    """One ionizing collision from a mono-energetic start (Eq. 9 with the
    ionization threshold as epsilon_k, then the uniform split of reading R9),
    against moments written from the equation, not from the oracle's code.
    With the new direction isotropic (cos theta uniform on [-1, 1]), the
    energy ratio is A + B cos theta, A = 1 - M/(m+M) x - 2mM/(m+M)^2,
    B = 2mM/(m+M)^2 sqrt(1 - (m+M)/M x), x = IP/eps0, and the primary keeps
    (1 - U) of it: E[eps'] = eps0 A / 2, E[eps'^2] = eps0^2 (A^2 + B^2/3) / 3,
    E[eps' cos theta] = eps0 B / 6.  A light target (M = 4 m) makes every
    term of Eq. 9 a visible share of the mean; a dropped term, a wrong sign of
    the angular term or a split other than a uniform fraction fails."""
    M_t, ip, eps0, n = 4 * ME, 15.0, 50.0, 200_000
    e = np.geomspace(ip, 1e4, 2001)
    v = np.sqrt(2 * e * QE / ME)
    nd = W.N_STP_293
    gas = W.Gas("ion4", M_t, nd, W.ISOTROPIC, [W.Channel(W.IONIZATION, ip, e, 1e12 / (nd * v))])
    m = O.Mixture([gas])
    rng = np.random.default_rng(77)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    speed = math.sqrt(2 * eps0 * QE / ME)
    state = np.zeros((n, 8))
    state[:, 3:6] = d * speed
    state[:, 7] = m.nu(eps0) * (1 + 1e-9)
    out, dec, eio = O.step_replay(m, state, np.arange(n, dtype=np.uint64), np.full(n, 5, np.uint32),
                                  e_over_n_Td=0.0, seed=2024)
    real = dec >= 0
    assert real.mean() > 0.999
    ef = 0.5 * ME * np.sum(out[real, 3:6] ** 2, axis=1) / QE
    vn = out[real, 3:6] / np.linalg.norm(out[real, 3:6], axis=1)[:, None]
    ct = np.sum(vn * d[real], axis=1)
    x = ip / eps0
    kappa = 2 * ME * M_t / (ME + M_t) ** 2
    A = 1 - M_t / (ME + M_t) * x - kappa
    B = kappa * math.sqrt(1 - x / (M_t / (ME + M_t)))
    for sample, expect in ((ef, eps0 * A / 2), (ef ** 2, eps0 ** 2 * (A * A + B * B / 3) / 3),
                           (ef * ct, eps0 * B / 6), (ct, 0.0), (ct ** 2, 1.0 / 3.0)):
        se = sample.std() / math.sqrt(len(sample))
        assert abs(sample.mean() - expect) < 4 * se, (sample.mean(), expect, se)


def test_isotropic_scattering_kinematics():
    """Isotropic elastic scattering (Sec. 2, Eq. 8) through the whole trial
    step: whatever the incident direction, the new one is uniform on the
    sphere, the cosine between incident and new direction is uniform on
    [-1, 1], and the energy kept is Eq. 8 at that measured cosine."""
    gas = _const_rate_gas(1e12)               # one elastic channel, isotropic, M = 1000 m
    mass = gas.mass_kg
    m = O.Mixture([gas])
    n = 100000
    eps = 5.0
    speed = math.sqrt(2 * eps * QE / ME)
    state = np.zeros((n, 8))
    state[:, 3] = speed                          # every electron comes in along +x
    state[:, 7] = m.nu(eps) * (1 + 1e-9)         # nearly every trial is real
    out, dec, eio = O.step_replay(m, state, np.arange(n, dtype=np.uint64), np.full(n, 7, np.uint32),
                                  e_over_n_Td=0.0, seed=17)
    real = dec >= 0
    assert real.mean() > 0.999
    vo = out[real, 3:6]
    so = np.linalg.norm(vo, axis=1)
    do = vo / so[:, None]
    k = real.sum()
    # uniform on the sphere: mean 0, second moments 1/3 (within 5 SE)
    assert np.all(np.abs(do.mean(axis=0)) < 5 * math.sqrt(1 / 3 / k))
    assert np.all(np.abs((do ** 2).mean(axis=0) - 1 / 3) < 5 * math.sqrt(4 / 45 / k))
    ct = do[:, 0]                                # cosine to the incident direction (+x)
    assert abs(ct.mean()) < 5 * math.sqrt(1 / 3 / k)
    # Eq. 8: E'/E = 1 - 2 m M / (m + M)^2 (1 - cos theta), at the measured angle
    kappa = 2 * ME * mass / (ME + mass) ** 2
    assert np.allclose((so / speed) ** 2, 1 - kappa * (1 - ct), rtol=1e-12, atol=0)


def test_fail_revert_and_fixed_mode():
    gases = [W.argon_like()]
    m = O.Mixture(gases)
    low = 0.3 * m.nu_max
    p = O.run_swarm(m, e_over_n_Td=300.0, real_collisions=200, n=200, seed=5, nu_trial=low, threads=4)
    assert p["n_fail"].sum() > 0
    assert np.all(p["n_real"] == 200)
    assert np.all(p["nu_p"] >= low)
    assert np.any(p["nu_p"] > low)
    q = O.run_swarm(m, e_over_n_Td=300.0, real_collisions=200, n=50, seed=5, nu_trial=low, fixed=True)
    assert np.all(q["status"][q["n_fail"] > 0] == O.ST_TRIAL)
    assert np.all(q["n_fail"] <= 1)


def test_time_limit_truncates_the_last_flight():
    m = O.Mixture([W.argon_like()])
    t_end = 2e-11
    p = O.run_swarm(m, e_over_n_Td=50.0, real_collisions=10 ** 6, n=100, seed=8, t_end=t_end)
    assert np.all(p["status"] == O.ST_TIME)
    assert np.all(p["t"] == t_end)


# --------------------------------------------------------------------------
# Swarm estimators and units, pinned by the worked example of Sec. 7.
# --------------------------------------------------------------------------
def test_worked_example_conventions():
    g = read_golden("drifter_example.txt")
    N = g["gas_density"] * 1e6                       # m^-3
    E = g["electric_field"] * 1e5                    # V/m
    W_ = g["drift_velocity"] * 1e4                   # m/s
    assert E / N / 1e-21 == pytest.approx(g["reduced_field"], rel=1e-5, abs=0.0)
    d = T.derived(W_, g["diffusion"] * 1e-4, g["diffusion_long"] * 1e-4, g["diffusion_tran"] * 1e-4,
                  E / N / 1e-21, N)
    assert d["mu"] * 1e4 == pytest.approx(g["mobility"], rel=1e-5, abs=0.0)
    assert d["mu_N"] * 1e-2 == pytest.approx(g["mobility_norm"], rel=1e-5, abs=0.0)
    assert d["mu_0"] * 1e4 == pytest.approx(g["mobility_reduced"], rel=1e-5, abs=0.0)
    assert d["D_over_mu"] == pytest.approx(g["diffusion_ratio"], rel=1e-5, abs=0.0)
    assert d["D_L_over_mu"] == pytest.approx(g["diffusion_long_ratio"], rel=1e-5, abs=0.0)
    assert d["D_T_over_mu"] == pytest.approx(g["diffusion_tran_ratio"], rel=1e-5, abs=0.0)
    assert d["ND"] * 1e-2 == pytest.approx(g["diffusion_norm"], rel=1e-5, abs=0.0)
    # D carries no 1/6: the printed D equals 2 D_L + 4 D_T to the printed digits
    assert 2 * g["diffusion_long"] + 4 * g["diffusion_tran"] == pytest.approx(g["diffusion"], abs=0.5)
    eff = 100 * T.efficiency(g["real_collisions"], g["null_collisions"], g["fail_collisions"])
    assert eff == pytest.approx(g["efficiency"], abs=5e-4)
    # N of the example is p / (k_B T) at 101.325 kPa, 293.15 K
    assert W.N_STP_293 == pytest.approx(N, rel=1e-5, abs=0.0)


def test_estimators_on_a_hand_worked_swarm():
    # two particles; W_vec = mean(x/t) = (0, 0, 3); d = x - t W_vec
    p = {"x": np.array([1.0, -2.0]), "y": np.array([0.0, 0.0]), "z": np.array([2.0, 8.0]),
         "t": np.array([1.0, 2.0]), "sum_e": np.array([10.0, 20.0]), "sum_e2": np.array([9.0, 18.0]),
         "n_real": np.array([10, 10]), "n_null": np.array([5, 5]), "n_fail": np.array([0, 0]),
         "n_ion": np.array([1, 0]), "n_att": np.array([0, 2]), "id": np.array([0, 1], dtype=np.uint64)}
    tr = T.swarm_tallies(p, 1.0, 1e25, groups=2)
    assert tr["W"] == 3.0 and tr["Wx"] == 0.0
    # d = (1, 0, -1) and (-2, 0, 2)
    assert tr["D"] == pytest.approx((2 / 1 + 8 / 2) / 2, abs=0.0)
    assert tr["D_L"] == pytest.approx((1 / 2 + 4 / 4) / 2, abs=0.0)
    assert tr["D_T"] == pytest.approx((1 / 4 + 4 / 8) / 2, abs=0.0)
    assert tr["D"] == pytest.approx(2 * tr["D_L"] + 4 * tr["D_T"], abs=0.0)
    assert tr["sig"] == pytest.approx((2 * math.sqrt(2) + 2 * math.sqrt(8)) / 2, abs=0.0)
    assert tr["sig_L"] == pytest.approx((2 + 4) / 2, abs=0.0)
    assert tr["sig_T"] == pytest.approx((2 + 4) / 2, abs=0.0)
    assert tr["alpha"] == pytest.approx((1 / 2 + 0) / 2, abs=0.0)
    assert tr["eta"] == pytest.approx((0 + 2 / 8) / 2, abs=0.0)
    assert tr["eps"] == pytest.approx(30 / 20, abs=0.0) and tr["eps_after"] == pytest.approx(27 / 20, abs=0.0)
    assert tr["efficiency"] == pytest.approx(20 / 30, abs=0.0)
    # with a transverse drift the full drift vector is taken out of d
    p["x"] = np.array([2.0, 2.0])
    tr = T.swarm_tallies(p, 1.0, 1e25, groups=2)
    assert tr["Wx"] == 1.5
    # d_x = 2 - 1.5 = 0.5 and 2 - 3 = -1
    assert tr["D_T"] == pytest.approx((0.25 / 4 + 1 / 8) / 2, abs=0.0)


# --------------------------------------------------------------------------
# Spawn mode: closed forms of constant-rate branching and removal.
# --------------------------------------------------------------------------
def _const_rate_gas(nu_el, nu_ion=0.0, nu_att=0.0):
    """sigma proportional to 1/v for each channel, so each rate is constant."""
    e = np.geomspace(1e-6, 1e4, 3001)
    v = np.sqrt(2 * e * QE / ME)
    n = W.N_STP_293
    ch = [W.Channel(W.ELASTIC, 0.0, e, nu_el / (n * v))]
    if nu_ion:
        ch.append(W.Channel(W.IONIZATION, 0.0, e, nu_ion / (n * v)))
    if nu_att:
        ch.append(W.Channel(W.ATTACHMENT, 0.0, e, nu_att / (n * v)))
    return W.Gas("const", 1000 * ME, n, W.ISOTROPIC, ch)


def test_spawn_population_grows_as_a_yule_process():
    nu_i = 1e11
    m = O.Mixture([_const_rate_gas(1e12, nu_ion=nu_i)])
    n0, t_end = 2000, 3.0 / nu_i
    p = O.run_swarm_spawn(m, e_over_n_Td=50.0, real_collisions=10 ** 9, n=n0, seed=21, pop_cap=200000, t_end=t_end)
    total = len(p["t"])
    expect = n0 * math.exp(nu_i * t_end)
    sd = math.sqrt(n0 * math.exp(nu_i * t_end) * (math.exp(nu_i * t_end) - 1))
    assert abs(total - expect) < 4 * sd
    assert np.all(p["status"] == O.ST_TIME)
    # one secondary per ionization, born inside the run, with the derived id
    assert total - n0 == int(p["n_ion"].sum())
    assert np.all(p["t_birth"][n0:] > 0) and np.all(p["t_birth"][n0:] < t_end)
    assert np.all(p["t_birth"] + p["t"] == pytest.approx(t_end, rel=1e-12, abs=0.0))
    assert len(np.unique(p["id"])) == total and np.all(p["id"][n0:] >= 2 ** 63)


def test_spawn_attachment_removes_at_a_constant_rate():
    nu_a = 1e11
    m = O.Mixture([_const_rate_gas(1e12, nu_att=nu_a)])
    n0, t_end = 20000, 1.5 / nu_a
    p = O.run_swarm_spawn(m, e_over_n_Td=10.0, real_collisions=10 ** 9, n=n0, seed=5, pop_cap=n0, t_end=t_end)
    alive = int(np.sum(p["status"] == O.ST_TIME))
    q = math.exp(-nu_a * t_end)
    assert abs(alive - n0 * q) < 4 * math.sqrt(n0 * q * (1 - q))
    removed = p["status"] == O.ST_ATTACHED
    assert np.all(p["n_att"][removed] == 1) and np.all(p["n_att"][~removed] == 0)


def test_secondary_ids_follow_the_splitmix64_finaliser():
    # SplitMix64 finaliser of parent * golden + step + 1, top bit set (written out here in integers)
    def mix(parent, step):
        z = (parent * 0x9E3779B97F4A7C15 + step + 1) & (2 ** 64 - 1)
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & (2 ** 64 - 1)
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & (2 ** 64 - 1)
        return (z ^ (z >> 31)) | 2 ** 63
    for parent, step in [(0, 0), (1, 7), (2 ** 40 + 3, 123456), (2 ** 63 + 9, 2 ** 32 - 1)]:
        assert O.secondary_id(parent, step) == mix(parent, step)


# --------------------------------------------------------------------------
# The paper's adaptive trial frequencies (Sec. 6.3 Binned, Sec. 6.4 Variable)
# --------------------------------------------------------------------------
def _sampled_max(m, gases, a, b, n=200001):
    """max of nu over [a, b] by dense sampling plus every table point inside."""
    xs = np.linspace(a, b, n)
    pts = [np.asarray(ch.energy_eV) for g in gases for ch in g.channels]
    inner = np.concatenate([p[(p >= a) & (p <= b)] for p in pts] + [xs])
    return float(m.nu_many(inner).max())


def test_range_max_matches_brute_force():
    rng = np.random.default_rng(17)
    for gases in ([W.argon_like()], W.ar_co2_mixture(), [W.batched_gases()[3], W.batched_gases()[5]]):
        m = O.Mixture(gases)
        for _ in range(12):
            a = float(10 ** rng.uniform(-3.5, 2.3))
            b = a * float(10 ** rng.uniform(0.01, 0.8))
            got, ref = m.range_max(a, b), _sampled_max(m, gases, a, b)
            # exact maximum: never below a sampled value, and the samples come close to it
            assert got >= ref * (1 - 1e-12)
            assert got <= ref * (1 + 2e-6)
        # a bin of BinnedTrialFrequency is the range [10^(j/B), 10^((j+1)/B))
        for B, j in ((8, -9), (8, 5), (3, 2), (1, 1)):
            assert m.binned_max(B, j) == m.range_max(10 ** (j / B), 10 ** ((j + 1) / B))


def _maxwell_run(**strategy):
    spec = W.maxwell_swarm(n_electrons=4000, real_collisions=600)
    gas = spec.gases[0]
    m = O.Mixture(spec.gases)
    p = O.run_swarm(m, e_over_n_Td=spec.e_over_n_Td, real_collisions=spec.real_collisions, n=spec.n_electrons,
                    seed=spec.seed, eps0_mean_eV=spec.eps0_mean_eV, threads=O.cpu_count(), **strategy)
    return spec, gas, m, p


def test_variable_trial_frequency_on_a_constant_frequency_gas():
    """With nu constant, nu' = (1 + zeta) nu never fails and the process is
    exact: the efficiency (Eq. 28) is 1/(1 + zeta) and the transport
    coefficients keep their closed forms."""
    zeta = 0.25
    spec, gas, m, p = _maxwell_run(strategy=O.TF_VARIABLE, zeta=zeta, grace=7)
    assert np.all(p["n_real"] == 600) and np.all(p["n_fail"] == 0)
    trials = p["n_real"].sum() + p["n_null"].sum()
    eff = p["n_real"].sum() / trials
    se = math.sqrt(eff * (1 - eff) / trials)
    assert abs(eff - 1 / (1 + zeta)) < 5 * se
    nu = 1e12
    E = spec.e_over_n_Td * 1e-21 * gas.number_density_m3
    vd = QE * E / (ME * nu)
    tr = T.swarm_tallies(p, spec.e_over_n_Td, gas.number_density_m3)
    assert abs(tr["W"] - vd) < 3.5 * tr["W_se"]
    kappa = 2 * ME * gas.mass_kg / (ME + gas.mass_kg) ** 2
    mean_eps, _, _ = _maxwell_closed_forms(600, 0.1, nu, kappa, vd)
    assert abs(tr["eps"] - mean_eps) < 3.5 * tr["eps_se"]


def test_binned_trial_frequency_on_a_constant_frequency_gas():
    """Bins of a constant-frequency gas all hold the same maximum (up to the
    table's interpolation ripple), so nu' = nu (1 + O(1e-5))."""
    spec, gas, m, p = _maxwell_run(strategy=O.TF_BINNED, bins_per_decade=8, grace=11)
    assert np.all(p["status"] == O.ST_DONE)
    eff = p["n_real"].sum() / (p["n_real"].sum() + p["n_null"].sum() + p["n_fail"].sum())
    assert eff > 0.9999
    E = spec.e_over_n_Td * 1e-21 * gas.number_density_m3
    vd = QE * E / (ME * 1e12)
    tr = T.swarm_tallies(p, spec.e_over_n_Td, gas.number_density_m3)
    assert abs(tr["W"] - vd) < 3.5 * tr["W_se"]


def _energy(p):
    return 0.5 * ME * (p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2) / QE


def test_adaptive_queries_follow_the_strategy_rules():
    """Grace counts null and real collisions alike (Sec. 6); with a grace of
    one, nu' is queried after every collision, so the last query happens
    right after the last real collision, at the energy the electron leaves
    with: Variable gives (1 + zeta) nu(eps), Binned the maximum over eps's bin."""
    gases = W.ar_co2_mixture()
    m = O.Mixture(gases)
    kw = dict(e_over_n_Td=20.0, real_collisions=60, n=300, seed=5, threads=O.cpu_count())
    p = O.run_swarm(m, strategy=O.TF_VARIABLE, zeta=0.4, grace=1, **kw)
    ok = p["status"] == O.ST_DONE
    eps = _energy(p)[ok]
    # floor: nu at the lowest positive table energy or threshold
    first = min(min(e for e in ch.energy_eV if e > 0) for g in gases for ch in g.channels)
    first = min([first] + [ch.threshold_eV for g in gases for ch in g.channels if ch.threshold_eV > 0])
    floor = max(1e-9 * m.nu_max, m.nu(first))
    want = 1.4 * np.maximum(m.nu_many(eps), floor)
    assert ok.sum() > 250
    assert np.allclose(p["nu_p"][ok], want, rtol=1e-12, atol=0.0)
    # Binned: whatever the grace, nu' is always one bin's maximum (a query
    # takes the bin of the current energy, a retry the larger of two bins)
    p = O.run_swarm(m, strategy=O.TF_BINNED, bins_per_decade=4, grace=25, max_trials=200000, **kw)
    assert (p["status"] == O.ST_DONE).sum() > 150
    maxima = {max(m.binned_max(4, j), floor) for j in range(-16, 12)}
    assert all(v in maxima for v in p["nu_p"])


def test_binned_second_fail_before_a_real_collision_is_an_error():
    """Sec. 6.3: after a fail the flight is retried with the larger of the two
    bins' maxima; if it fails again the run stops with an error.  With one
    bin per decade at a strong field, electrons cross bins often."""
    m = O.Mixture([W.argon_like()])
    p = O.run_swarm(m, e_over_n_Td=300.0, real_collisions=400, n=400, seed=8, threads=O.cpu_count(),
                    strategy=O.TF_BINNED, bins_per_decade=1, grace=1000, max_trials=200000)
    err = p["status"] == O.ST_TRIAL
    assert err.any() and (~err).any()
    assert np.all(p["n_fail"][err] >= 2)
    # every nu' left behind is one bin's maximum (a retry takes the larger of two)
    floor = m.nu(1e-3)   # nu at the lowest table energy
    maxima = {max(m.binned_max(1, j), floor) for j in range(-6, 6)}
    assert all(v in maxima for v in p["nu_p"])


def test_invalid_strategies_are_rejected():
    m = O.Mixture([W.argon_like()])
    kw = dict(e_over_n_Td=10.0, real_collisions=5, n=4, seed=1)
    for bad in (dict(strategy=O.TF_VARIABLE, zeta=-0.1), dict(strategy=O.TF_BINNED, bins_per_decade=0),
                dict(strategy=O.TF_VARIABLE, grace=0), dict(strategy=7)):
        with pytest.raises(ValueError):
            O.run_swarm(m, **kw, **bad)


# --------------------------------------------------------------------------
# xi form of the scattering angle for non-polar molecules (Eqs. 6-7)
# --------------------------------------------------------------------------
def test_xi_form_mean_deflection_is_the_cross_section_ratio():
    """The xi form is built so that the mean of 1 - cos(theta) under Eq. 6
    equals sigma_mt / sigma_el, the right side of Eq. 7 (substituting
    u = 1 + xi - 2 xi R makes the integral elementary).  Quadrature of the
    sampler over R therefore pins both equations against each other."""
    from scipy import integrate
    for xi in (-0.95, -0.6, -0.2, -0.01, 0.003, 0.04, 0.06, 0.3, 0.7, 0.95, 0.999):
        mean, err = integrate.quad(lambda R: 1.0 - O.cos_theta_xi(xi, R), 0.0, 1.0, epsabs=0.0, epsrel=1e-12,
                                   limit=200)
        assert O.xi_ratio(xi) == pytest.approx(mean, rel=1e-10, abs=0.0), xi


def test_xi_form_limits():
    # isotropic at xi = 0; the ratio falls monotonically from 2 (backward) to 0 (forward)
    for R in (0.0, 0.1, 0.5, 0.9):
        assert O.cos_theta_xi(0.0, R) == 1.0 - 2.0 * R
    assert O.xi_ratio(0.0) == 1.0
    xs = np.linspace(-0.999, 0.999, 2001)
    r = np.array([O.xi_ratio(x) for x in xs])
    assert np.all(np.diff(r) < 0) and r[0] < 2.0 and r[-1] > 0.0
    assert O.xi_ratio(-1 + 1e-12) == pytest.approx(2.0, abs=1e-9)
    assert O.xi_ratio(1 - 1e-12) == pytest.approx(0.0, abs=1e-9)
    # the series (|xi| < 0.05) and the closed form meet smoothly
    assert O.xi_ratio(0.0499999) == pytest.approx(O.xi_ratio(0.0500001), abs=1e-6)
    # every cos(theta) is a cosine
    for xi in (-0.99, -0.5, 0.5, 0.99):
        c = [O.cos_theta_xi(xi, R) for R in np.linspace(0.0, 1.0, 101)]
        assert min(c) >= -1.0 - 1e-12 and max(c) <= 1.0 + 1e-12


def test_xi_solve_and_gas_xi():
    for r in (1e-4, 0.05, 0.4, 0.999, 1.0, 1.3, 1.9, 1.9999):
        xi = O.xi_solve(r)
        assert O.xi_ratio(xi) == pytest.approx(r, rel=1e-12, abs=1e-14)
    assert abs(O.xi_solve(1.0)) < 1e-15
    # the xi-form CO2-like gas: sigma_el = sigma_mt (1 + eps / 5 eV), so r = 1 / (1 + eps / 5)
    gases = [W.argon_like(0.9 * W.N_STP_293), W.co2_like(0.1 * W.N_STP_293, xi_form=True)]
    m = O.Mixture(gases)
    # the table points of both cross sections coincide, so the ratio is exact at them
    grid = gases[1].sigma_el[0]
    for eps in (grid[0], grid[137], grid[350], grid[-1]):
        assert O.xi_ratio(m.gas_xi(1, eps)) == pytest.approx(1.0 / (1.0 + eps / 5.0), rel=1e-9, abs=0.0)
    # below the tables both extend with their first values (Sec. 2.2)
    assert m.gas_xi(1, 1e-5) == m.gas_xi(1, grid[0])
    assert m.gas_xi(0, 3.0) == 0.0            # argon has no total elastic table: isotropic


def test_xi_gas_with_equal_cross_sections_scatters_isotropically():
    """sigma_el = sigma_mt gives xi = 0, where Eq. 6 is the isotropic law
    (exact: test_xi_form_limits).  The isotropic gas draws its new direction
    in the lab frame and the xi gas turns the incident one, so the two swarms
    agree in distribution, not draw for draw: every one of their statistics
    within 3.5 combined standard errors (32 batch groups), and the null and
    real collision counts, which do not depend on the angle before the first
    real collision, identical for every electron's first flight."""
    base = W.co2_like()
    grid, s_mt = base.channels[0].energy_eV, base.channels[0].sigma_m2
    xi_gas = W.Gas("co2-xi-iso", base.mass_kg, base.number_density_m3, W.XI_FORM, base.channels,
                   sigma_el=(grid, s_mt))
    m_iso, m_xi = O.Mixture([base]), O.Mixture([xi_gas])
    kw = dict(e_over_n_Td=40.0, real_collisions=200, n=4000, seed=9, threads=O.cpu_count())
    a = T.swarm_tallies(O.run_swarm(m_iso, **kw), 40.0, m_iso.n_total)
    b = T.swarm_tallies(O.run_swarm(m_xi, **kw), 40.0, m_xi.n_total)
    for k in ("W", "eps", "eps_after", "D_L", "D_T"):
        assert abs(a[k] - b[k]) <= 3.5 * math.hypot(a[k + "_se"], b[k + "_se"]), (k, a[k], b[k])
    one = dict(kw, real_collisions=1, n=2000)
    p, q = O.run_swarm(m_iso, **one), O.run_swarm(m_xi, **one)
    for k in ("n_real", "n_null", "steps"):
        assert np.array_equal(p[k], q[k]), k
    assert np.allclose(p["z"], q["z"], rtol=1e-12, atol=1e-18)


def test_xi_form_forward_scattering_raises_the_drift_velocity():
    """Where sigma_el > sigma_mt the xi form scatters forward (xi > 0): with
    the momentum-transfer cross section fixed, forward scattering keeps more
    of the momentum gained from the field, so electrons drift at least as
    fast as with isotropic scattering (a sanity check, not a closed form)."""
    kw = dict(e_over_n_Td=60.0, real_collisions=300, n=3000, seed=12, threads=O.cpu_count())
    iso = O.run_swarm(O.Mixture([W.co2_like()]), **kw)
    fwd = O.run_swarm(O.Mixture([W.co2_like(xi_form=True)]), **kw)
    ti = T.swarm_tallies(iso, 60.0, W.N_STP_293)
    tf = T.swarm_tallies(fwd, 60.0, W.N_STP_293)
    assert tf["W"] > ti["W"] - 3 * math.hypot(ti["W_se"], tf["W_se"])


# --------------------------------------------------------------------------
# Moving targets (Sec. 2.1): collisions in the centre-of-momentum frame
# --------------------------------------------------------------------------
KB = 1.380649e-23


def test_thermal_collision_conserves_momentum_and_energy():
    rng = np.random.default_rng(5)
    for M_over_m in (1.0, 10.0, 7.3e4):
        m, M = ME, ME * M_over_m
        for eps_k in (0.0, 0.4):
            v1 = rng.normal(0, 1e6, 3)
            v2 = rng.normal(0, 3e3, 3)
            ct, phi = float(rng.uniform(-1, 1)), float(rng.uniform(0, 2 * math.pi))
            a, b = O.thermal_collide(v1, v2, m, M, eps_k, ct, phi)
            p0, p1 = m * v1 + M * v2, m * a + M * b
            assert np.allclose(p1, p0, rtol=0, atol=1e-12 * np.abs(p0).max())
            e0 = 0.5 * m * v1 @ v1 + 0.5 * M * v2 @ v2
            e1 = 0.5 * m * a @ a + 0.5 * M * b @ b
            assert e1 == pytest.approx(e0 - eps_k * QE, rel=1e-12, abs=0.0)
            # the centre-of-momentum frame turns the bullet by theta
            vcm = p0 / (m + M)
            g0, g1 = v1 - vcm, a - vcm
            assert g0 @ g1 / (np.linalg.norm(g0) * np.linalg.norm(g1)) == pytest.approx(ct, abs=1e-12)


def _thermal_gas():
    # constant collision frequency nu = 1e12/s, target mass 10 m (light, so the mass factors show)
    return W.maxwell_gas(nu=1e12, mass_ratio=0.1)


def test_thermal_equilibrium_at_zero_field():
    """Without a field, electrons among targets at temperature T relax to the
    Maxwellian at T (a constant collision frequency keeps detailed balance):
    mean energy 3/2 kT, energies distributed as Gamma(3/2, kT)."""
    temp = 293.15
    kT = KB * temp / QE
    m = O.Mixture([_thermal_gas()])
    p = O.run_swarm(m, e_over_n_Td=0.0, real_collisions=300, n=6000, seed=17, threads=O.cpu_count(), gas_T=temp)
    eps = 0.5 * ME * (p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2) / QE
    assert abs(eps.mean() - 1.5 * kT) < 4 * eps.std() / math.sqrt(len(eps))
    assert stats.kstest(eps / kT, stats.gamma(1.5).cdf).pvalue > 1e-3
    # targets at rest instead: the electrons keep cooling (20 collisions take
    # the 0.1 eV start to ~3 meV, well below 3/2 kT)
    q = O.run_swarm(m, e_over_n_Td=0.0, real_collisions=20, n=2000, seed=17, threads=O.cpu_count())
    assert (0.5 * ME * (q["vx"] ** 2 + q["vy"] ** 2 + q["vz"] ** 2) / QE).mean() < 0.5 * kT


def thermal_expectations(I, eps0_eV, nu, E, M, temp):
    """Exact means for a constant collision frequency, isotropic scattering in
    the centre-of-momentum frame and targets at temperature T, started from
    an isotropic distribution of mean energy eps0 (zero mean velocity).  Per
    collision the mean velocity becomes m/(m+M) of its value (the target's
    mean is 0, the centre-of-momentum velocity keeps the rest) and
    <eps'> = (1 - kappa) eps + kappa 3/2 kT, kappa = 2 m M / (m + M)^2; an
    exponential flight of mean 1/nu from velocity u adds u/nu + a/nu^2 to z
    and m a u / nu + m a^2 / nu^2 to the energy (<tau^2> = 2/nu^2).  Returns
    (E[sum z] / E[sum t], mean energy before a collision [eV]); their steady
    states are v_d = eE/(mu nu) and 3/2 kT + (eE)^2/(mu nu^2 kappa)."""
    a = QE * E / ME
    b = ME / (ME + M)
    kappa = 2 * ME * M / (ME + M) ** 2
    u, ea, Z, eb_sum = 0.0, eps0_eV * QE, 0.0, 0.0
    for _ in range(I):
        Z += u / nu + a / nu ** 2
        eb = ea + ME * a * u / nu + ME * a * a / nu ** 2
        eb_sum += eb
        u = b * (u + a / nu)
        ea = (1 - kappa) * eb + kappa * 1.5 * KB * temp
    return Z / (I / nu), eb_sum / I / QE


def test_thermal_drift_and_mean_energy_closed_forms():
    """Constant collision frequency, isotropic scattering in the centre-of-
    momentum frame, targets at T: momentum balance gives v_d = eE/(mu nu)
    (mu the reduced mass); per collision <d eps> = -kappa (eps - 3/2 kT) with
    kappa = 2 m M / (m + M)^2, so <eps> = 3/2 kT + (eE)^2 / (mu nu^2 kappa).
    The ratio-of-sums drift and the collision-averaged energy are compared
    with the exact means of the transient from the start (above)."""
    temp, nu = 293.15, 1e12
    gas = _thermal_gas()
    M = gas.mass_kg
    mu, kappa = ME * M / (ME + M), 2 * ME * M / (ME + M) ** 2
    eon = 10.0
    E = eon * 1e-21 * gas.number_density_m3
    p = O.run_swarm(O.Mixture([gas]), e_over_n_Td=eon, real_collisions=1000, n=6000, seed=19,
                    threads=O.cpu_count(), gas_T=temp)
    t = OT_tallies(p, eon, gas.number_density_m3)
    vd = QE * E / (mu * nu)
    mean_eps = 1.5 * KB * temp / QE + (QE * E) ** 2 / (mu * nu ** 2 * kappa) / QE
    w_exp, e_exp = thermal_expectations(1000, 0.1, nu, E, M, temp)
    assert w_exp == pytest.approx(vd, rel=2e-3, abs=0.0) and e_exp == pytest.approx(mean_eps, rel=2e-3, abs=0.0)
    assert abs(t["W_flux"] - w_exp) < 3.5 * t["W_se"]
    assert abs(t["eps"] - e_exp) < 3.5 * t["eps_se"]
    # and the mass factor matters: the heavy-target formula is several SE away
    assert abs(t["W_flux"] - QE * E / (ME * nu)) > 5 * t["W_se"]


def OT_tallies(p, eon, n):
    return T.swarm_tallies(p, eon, n)
