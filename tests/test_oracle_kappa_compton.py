"""Pins of the oracle's Compton scattering off kappa-distributed electrons (the kappa population of
section 6 carried into the Klein-Nishina kinematics of section 2.7):

* the hot cross-section table against a direct two-dimensional quadrature (scipy, in gamma and mu), the
  Thomson limit sigma_h -> sigma_T, and the kappa -> infinity limit, where the population becomes
  Maxwell-Juettner at Theta = w and the table must reproduce the thermal cross-section;
* the Lorentz-factor sampler against the kappa density, bin by bin, from kappa = 3.1 (envelope terms
  with shape below 1) to kappa = 1e5 (the thermal limit), on both sides of the w = 1 envelope switch;
* the scattered photon in the Thomson limit: mean energy gain 1 + (4/3) <gamma^2 beta^2> with <.>
  over the kappa density (no recoil at eps = 1e-10), and the forward-backward symmetric angular law of
  a slow population.
"""
import numpy as np
import pytest
from scipy import integrate

SIGMA_T = 6.6524587321e-25


def kappa_logpdf(kap, w):
    kw = kap * w
    return lambda g: np.log(g) + 0.5 * np.log(g * g - 1.0) - (kap + 1.0) * np.log1p((g - 1.0) / kw)


def kappa_cdf_mass(kap, w, a, b, ref):
    lf = kappa_logpdf(kap, w)
    return integrate.quad(lambda g: np.exp(lf(g) - ref), a, b, limit=400, epsrel=1e-10)[0]


def kappa_norm(kap, w, ref):
    pts = [1.0, 1.0 + w, 1.0 + 10.0 * w, 1.0 + 1e3 * w]
    s = sum(kappa_cdf_mass(kap, w, a, b, ref) for a, b in zip(pts[:-1], pts[1:]))
    return s + kappa_cdf_mass(kap, w, pts[-1], np.inf, ref)


def sigma_hot_direct(oracle_mod, kap, w, eps):
    """<(1 - beta mu) sigma_KN(eps gamma (1 - beta mu))> / sigma_T over the kappa density, scipy in t = ln(gamma - 1)."""
    lf = kappa_logpdf(kap, w)
    ref = lf(1.0 + w)

    def dens(t):
        g = 1.0 + np.exp(t)
        return np.exp(lf(g) - ref) * np.exp(t)

    def inner(t):
        g = 1.0 + np.exp(t)
        beta = np.sqrt(1.0 - 1.0 / (g * g))
        return 0.5 * integrate.quad(lambda mu: (1 - beta * mu) * oracle_mod.sigma_kn(eps * g * (1 - beta * mu)),
                                    -1.0, 1.0, epsabs=0.0, epsrel=1e-11, limit=200)[0]

    t0, t1 = np.log(kap * w) - 25.0, np.log(kap * w) + 45.0
    brk = list(np.log(w) + np.arange(-6.0, 12.0, 1.0))
    num = integrate.quad(lambda t: dens(t) * inner(t), t0, t1, points=brk, limit=400, epsabs=0.0, epsrel=1e-9)[0]
    den = integrate.quad(dens, t0, t1, points=brk, limit=400, epsrel=1e-11)[0]
    return num / den / SIGMA_T


@pytest.mark.parametrize("kap,iw,ie", [(4.0, 30, 120), (3.5, 10, 150), (10.0, 45, 100), (4.0, 60, 120)])
def test_hot_table_node_matches_direct_quadrature(oracle_mod, kap, iw, ie):
    # table nodes: ln w on [ln 1e-3, ln 1e3] (61 nodes), ln eps on [ln 1e-12, ln 1e6] (181 nodes)
    w = np.exp(np.log(1e-3) + (np.log(1e3) - np.log(1e-3)) * iw / 60)
    eps = np.exp(np.log(1e-12) + (np.log(1e6) - np.log(1e-12)) * ie / 180)
    tab = oracle_mod.sigma_hot_kappa(kap, w, eps) / SIGMA_T
    ref = sigma_hot_direct(oracle_mod, kap, w, eps)
    assert abs(tab / ref - 1.0) < 2e-6, (tab, ref)


@pytest.mark.parametrize("kap", [3.2, 4.0, 20.0])
def test_hot_table_thomson_limit(oracle_mod, kap):
    for w in (1e-3, 0.1, 1.0, 10.0, 300.0):
        assert abs(oracle_mod.sigma_hot_kappa(kap, w, 1e-12) / SIGMA_T - 1.0) < 1e-6
    # and it falls with photon energy
    v = [oracle_mod.sigma_hot_kappa(kap, 1.0, e) for e in (1e-6, 1e-3, 1e-1, 1.0, 10.0, 1e3)]
    assert np.all(np.diff(v) < 0.0)


def test_hot_table_thermal_limit(oracle_mod):
    kap = 1e5
    for th in (0.01, 0.1, 1.0, 10.0):
        for eps in (1e-4, 1e-2, 1.0, 30.0):
            # (1 + (gamma - 1) / (kappa w))^-(kappa+1) -> exp(-(gamma - 1) / w): Maxwell-Juettner at Theta = w
            r = oracle_mod.sigma_hot_kappa(kap, th, eps) / oracle_mod.sigma_hot_quad(th, eps)
            assert abs(r - 1.0) < 3e-4, (th, eps, r)


@pytest.mark.parametrize("kap,w", [(3.1, 0.01), (3.1, 30.0), (4.0, 0.5), (4.0, 1.0), (8.0, 2.0), (1e5, 0.02),
                                   (1e5, 3.0), (50.0, 100.0)])
def test_sampler_matches_density(oracle_mod, kap, w):
    n = 100000
    g = oracle_mod.sample_kappa(kap, w, n, seed=7, stream=int(kap * 10 + w * 100))
    assert np.all(g >= 1.0) and np.all(np.isfinite(g))
    ref = kappa_logpdf(kap, w)(1.0 + w)
    Z = kappa_norm(kap, w, ref)
    edges = np.quantile(g, [0.0, 0.05, 0.2, 0.4, 0.6, 0.8, 0.95, 0.999])
    edges[0] = 1.0
    for a, b in zip(edges[:-1], edges[1:]):
        p = kappa_cdf_mass(kap, w, a, b, ref) / Z
        o = np.mean((g >= a) & (g < b))
        assert abs(o - p) < 5.0 * np.sqrt(p * (1 - p) / n), (a, b, o, p)


def test_thomson_energy_gain(oracle_mod):
    kap, w = 8.0, 0.3          # <gamma^4> finite for kappa > 6: the sample mean has a finite variance
    th = w * kap / (kap - 3.0)
    ref = kappa_logpdf(kap, w)(1.0 + w)
    Z = kappa_norm(kap, w, ref)
    lf = kappa_logpdf(kap, w)
    m = sum(integrate.quad(lambda g: np.exp(lf(g) - ref) * (g * g - 1.0), a, b, limit=400)[0]
            for a, b in [(1.0, 1.0 + w), (1.0 + w, 1.0 + 10 * w), (1.0 + 10 * w, np.inf)]) / Z
    eps = 1e-10
    eo, mu = oracle_mod.compton_kappa(kap, th, eps, 200000, seed=9)
    r = eo / eps
    assert abs(np.mean(r) - (1.0 + 4.0 / 3.0 * m)) < 5.0 * np.std(r) / np.sqrt(len(r))
    assert np.all(np.abs(mu) <= 1.0 + 1e-12)


def test_slow_population_scatters_like_thomson(oracle_mod):
    # w = 1e-3 with large kappa: electrons nearly at rest, the angular law is (1 + mu^2) (3/8) and the energy
    # is unchanged to O(sqrt(w))
    eo, mu = oracle_mod.compton_kappa(1e4, 1e-3, 1e-9, 100000, seed=4)
    assert abs(np.mean(mu)) < 5 * np.sqrt(0.4 / len(mu))
    assert abs(np.mean(mu * mu) - 0.4) < 5 * np.sqrt(0.1 / len(mu))
    assert abs(np.median(eo / 1e-9) - 1.0) < 0.05
