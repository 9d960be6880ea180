"""Oracle pins of the kappa-electron synchrotron emission and absorption (future work in section 6):
the synchrotron function against its definition by scipy's Bessel K_5/3 and its textbook maximum,
the thermal limit (kappa -> infinity: the exact thermal emissivity and the paper's fit, eq.
emissivity), Kirchhoff's law alpha B_nu = j in that limit (a check of the absorption integral
against the emission one), and the power-law tail j ~ nu^-(kappa-2)/2 of a kappa population."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_2602_13198_gb300 import synth

EE, ME, CL = 4.803204712570263e-10, 9.1093837015e-28, 2.99792458e10


def F_scipy(x):
    f = lambda s: special.kv(5 / 3, x * math.exp(s)) * x * math.exp(s)
    return x * integrate.quad(f, 0, math.log1p(60 / x), limit=400, epsrel=1e-12)[0]


def j_thermal_exact(nu, ne, th, B):
    """Thermal synchrotron emissivity at 90 degrees to the field from the single-electron spectrum
    integrated over the Maxwell-Juettner distribution (scipy quadrature)."""
    nuB = EE * B / (2 * math.pi * ME * CL)
    pdf = lambda g: g * math.sqrt(g * g - 1) * math.exp(-g / th) / (th * special.kv(2, 1 / th))
    f = lambda lg: (lambda g: pdf(g) * F_scipy(nu / (1.5 * g * g * nuB)) * g)(math.exp(lg))
    return math.sqrt(3) * EE ** 3 * ne * B / (4 * math.pi * ME * CL * CL) * integrate.quad(f, 0, 12, limit=400)[0]


def j_fit(nu, ne, th, B):
    nus = (2 / 9) * (EE * B / (2 * math.pi * ME * CL)) * th * th
    X = nu / nus
    return math.sqrt(2) * math.pi * EE ** 2 * ne * nus / (3 * CL * special.kv(2, 1 / th)) * (
        X ** 0.5 + 2 ** (11 / 12) * X ** (1 / 6)) ** 2 * math.exp(-X ** (1 / 3))


def test_synchrotron_function():
    import oracle
    for x in (1e-6, 1e-3, 0.29, 1.0, 5.0):
        assert abs(oracle.F_sync(x) / F_scipy(x) - 1.0) < 1e-9, x
    xs = np.linspace(0.2, 0.4, 81)
    F = [oracle.F_sync(x) for x in xs]
    assert abs(xs[int(np.argmax(F))] - 0.29) < 0.01 and abs(max(F) - 0.918) < 1e-3


@pytest.fixture(scope="module")
def thermal_limit():
    p, _ = synth.sphere("flat", R=1.0, kappa=1e6)
    return p


def test_thermal_limit_matches_exact_and_fit(thermal_limit):
    import oracle
    th, B, ne = 10.0, 10.0, 1e13
    for nu in (1e10, 1e11, 1e12):
        jk = oracle.jnu_kappa(thermal_limit, nu, ne, th, B, 0.0)
        assert abs(jk / j_thermal_exact(nu, ne, th, B) - 1.0) < 3e-3
        assert abs(jk / j_fit(nu, ne, th, B) - 1.0) < 0.03


def test_kirchhoff_in_the_thermal_limit(thermal_limit):
    import oracle
    th, B, ne = 10.0, 10.0, 1e13
    for nu in (1e10, 1e12, 1e13):
        for c in (0.0, 0.6):
            j = oracle.jnu_kappa(thermal_limit, nu, ne, th, B, c)
            a = oracle.nu_alpha_kappa(thermal_limit, nu, ne, th, B, c) / nu
            assert abs(a * oracle.bnu(nu, th) / j - 1.0) < 2e-3


def test_power_law_tail():
    import oracle
    for kap in (3.5, 4.0, 6.0):
        p, _ = synth.sphere("flat", R=1.0, kappa=kap)
        j1, j2 = (oracle.jnu_kappa(p, 10 ** l, 1e13, 10.0, 10.0, 0.0) for l in (14.5, 15.0))
        slope = math.log(j2 / j1) / (0.5 * math.log(10))
        assert abs(slope + (kap - 2) / 2) < 0.03 * (kap - 2) / 2 + 0.01, (kap, slope)
