"""Oracle pins: Klein-Nishina and hot cross-sections, the Maxwell-Juettner and
Klein-Nishina samplers, and thermal Comptonisation in the Thomson limit (section 2.7)."""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

SIGMA_T = 6.6524587321e-25


def kn_diff(e, mu):
    """Klein-Nishina d sigma / d Omega / sigma_T (r_e^2 / 2 = 3 sigma_T / 16 pi)."""
    r = 1.0 / (1.0 + e * (1.0 - mu))
    return 3.0 / (16.0 * math.pi) * r * r * (r + 1.0 / r - (1.0 - mu * mu))


@pytest.mark.parametrize("e", [1.1e-3, 0.01, 0.3, 1.0, 10.0, 1e3])
def test_sigma_kn_vs_differential_integral(oracle_mod, e):
    ref, _ = integrate.quad(lambda mu: 2 * math.pi * kn_diff(e, mu), -1, 1, epsrel=1e-13, epsabs=0)
    assert oracle_mod.sigma_kn(e) / SIGMA_T == pytest.approx(ref, rel=1e-8)


def test_sigma_kn_thomson_series(oracle_mod):
    for e in (1e-8, 1e-5, 9e-4):
        ref, _ = integrate.quad(lambda mu: 2 * math.pi * kn_diff(e, mu), -1, 1, epsrel=1e-13, epsabs=0)
        assert oracle_mod.sigma_kn(e) / SIGMA_T == pytest.approx(1 - 2 * e, rel=1e-12)
        assert oracle_mod.sigma_kn(e) / SIGMA_T == pytest.approx(ref, rel=6e-6)


def mj_pdf(g, th):
    return g * g * math.sqrt(1 - 1 / (g * g)) * math.exp(-g / th) / (th * special.kv(2, 1 / th))


def mj_pdf_scaled(g, th):
    # e^{(1-g)/th} / (th K2e) with K2e = K2(1/th) e^{1/th}, safe for small th
    return g * g * math.sqrt(1 - 1 / (g * g)) * math.exp((1 - g) / th) / (th * special.kve(2, 1 / th))


def sigma_hot_ref(th, e):
    """Definition of the hot cross-section written with an adaptive 2-D quadrature."""
    def inner(g):
        b = math.sqrt(1 - 1 / (g * g))
        q, _ = integrate.quad(lambda mu: (1 - mu * b) * kn_sigma(e * g * (1 - mu * b)), -1, 1, epsrel=1e-11)
        return 0.5 * q
    gmax = 1 + 80 * th
    v, _ = integrate.quad(lambda g: mj_pdf_scaled(g, th) * inner(g), 1, gmax, epsrel=1e-9, limit=200)
    return v


def kn_sigma(e):
    if e < 1e-6:
        return 1 - 2 * e
    ref = 0.75 / e**2 * (2 + e * e * (1 + e) / (1 + 2 * e) ** 2 + (e * e - 2 * e - 2) / (2 * e) * math.log1p(2 * e))
    return ref


@pytest.mark.parametrize("th,e", [(0.5, 0.1), (4.0, 1e-2), (10.0, 1.0), (0.05, 3.0)])
def test_sigma_hot_quadrature_vs_definition(oracle_mod, th, e):
    assert oracle_mod.sigma_hot_quad(th, e) / SIGMA_T == pytest.approx(sigma_hot_ref(th, e), rel=1e-6)


def test_sigma_hot_limits(oracle_mod):
    # Thomson limit: for eps -> 0 the hot cross-section is sigma_T at any temperature
    for th in (1e-3, 0.3, 10.0, 1000.0):
        assert oracle_mod.sigma_hot_quad(th, 1e-12) / SIGMA_T == pytest.approx(1.0, rel=1e-6)
    # cold limit: Theta -> 0 gives the Klein-Nishina value of an electron at rest
    for e in (0.01, 1.0, 100.0):
        assert oracle_mod.sigma_hot_quad(1e-4, e) == pytest.approx(oracle_mod.sigma_kn(e), rel=2e-3)


def test_sigma_hot_table_interpolation(oracle_mod):
    rng = np.random.default_rng(5)
    for _ in range(20):
        th = math.exp(rng.uniform(math.log(2e-3), math.log(500.0)))
        e = math.exp(rng.uniform(math.log(1e-11), math.log(1e5)))
        assert oracle_mod.sigma_hot_table(th, e) == pytest.approx(oracle_mod.sigma_hot_quad(th, e), rel=2e-2)


@pytest.mark.parametrize("th", [0.03, 0.2, 0.25, 1.0, 4.0, 100.0])
def test_mj_sampler(oracle_mod, th):
    n = 40000
    g = oracle_mod.sample_mj(th, n, seed=11, stream=int(th * 1000))
    # closed-form mean <gamma> = K1(1/th)/K2(1/th) + 3 th
    mean = special.kve(1, 1 / th) / special.kve(2, 1 / th) + 3 * th
    sd = math.sqrt(np.var(g) / n)
    assert abs(g.mean() - mean) < 4 * sd
    # Kolmogorov-Smirnov against the exact CDF
    qs = np.quantile(g, np.linspace(0.05, 0.95, 19))
    cdf_at = np.array([integrate.quad(lambda x: mj_pdf_scaled(x, th), 1, q, epsrel=1e-10, limit=200)[0] for q in qs])
    emp = np.linspace(0.05, 0.95, 19)
    assert np.max(np.abs(cdf_at - emp)) < 1.63 / math.sqrt(n) * 2.0


@pytest.mark.parametrize("e", [1e-6, 1.0])
def test_kn_angle_sampler_cold_electrons(oracle_mod, e):
    n = 60000
    th = 1e-10   # electrons essentially at rest
    eo, d = oracle_mod.compton(th, e, n, seed=3, stream0=1000)
    mu = d[:, 2] / np.linalg.norm(d, axis=1)
    # per-event energy: eps' = eps / (1 + eps (1 - cos)) (electron at rest)
    assert np.allclose(eo, e / (1 + e * (1 - mu)), rtol=1e-4)
    edges = np.linspace(-1, 1, 21)
    h, _ = np.histogram(mu, bins=edges)
    tot, _ = integrate.quad(lambda m: kn_diff(e, m), -1, 1)
    p = np.array([integrate.quad(lambda m: kn_diff(e, m), edges[i], edges[i + 1])[0] / tot for i in range(20)])
    chi2 = ((h - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, 19) > 1e-3


@pytest.mark.parametrize("th", [0.1, 1.0, 4.0])
def test_thermal_thomson_mean_gain(oracle_mod, th):
    # Thomson limit, isotropic thermal electrons: <eps1/eps> = 1 + 4/3 <(gamma beta)^2>_MJ
    n = 100000
    eo, _ = oracle_mod.compton(th, 1e-9, n, seed=5, stream0=7)
    r = eo / 1e-9
    p2, _ = integrate.quad(lambda g: mj_pdf_scaled(g, th) * (g * g - 1), 1, 1 + 80 * th, epsrel=1e-11, limit=200)
    ref = 1 + 4.0 / 3.0 * p2
    assert abs(r.mean() - ref) < 4 * r.std() / math.sqrt(n)
