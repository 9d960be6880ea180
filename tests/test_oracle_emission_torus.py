"""Pin of the oracle's emission on moving, magnetised plasma (sections 2.1-2.3): the weights, zone
counts and frequency sampling on spinning tori against the emitted photon number and power computed
here from the zone volumes and the thermal synchrotron emissivity, without the oracle's weight
table, counts or sampler.

For zone i the expected count is n_i = V_i / h * int g_lin dln(nu) (g_lin the piecewise-linear
interpolant of int dOmega j_nu / w over the weight-table nodes), a superphoton's frequency is drawn
from g_lin and its weight is int dOmega j_nu(nu) / g_lin(nu).  So, whatever the table,
    E[sum of birth weights]         = sum_i V_i / h * int dOmega j_nu dln(nu)    (photons per unit time)
    E[sum of weight x h nu_fluid]   = sum_i V_i * int dOmega j_nu dnu             (emitted power),
over the table's frequency range.  The right-hand sides are computed here: volumes from sqrt(-g) of
modified Kerr-Schild coordinates, n_e, Theta_e and |B| at the zone centres from the oracle's fluid
state (pinned on its own in test_oracle_fluid), the angle-integrated emissivity from the paper's
fit with scipy's K_2 and numpy's Gauss-Legendre nodes, and integrals on a fine ln(nu) grid.  The
fluid-frame frequency of each birth wavevector is -k.u with the oracle's metric.  A dropped 1/h, a
weight without the g_lin correction, a count or volume off by a Jacobian, or a sampler that does
not follow g_lin fails one of the two."""
import math

import numpy as np
import pytest
from scipy import special

from paper_2602_13198_gb300 import synth

EE, ME, CL, HPL = 4.803204712570263e-10, 9.1093837015e-28, 2.99792458e10, 6.62607015e-27


def angle_integrated_jnu(nu, ne, th, B, k2_mode):
    """int dOmega j_nu of thermal synchrotron (section 2.2 fit): 4 pi A nu_c F(nu / nu_c),
    A = sqrt2 pi e^2 n_e / (3 c K2(1/Theta)), nu_c = (2/9) nu_B Theta^2, F(K) = int_0^{pi/2} sin^2 G(K / sin)."""
    xg, wg = np.polynomial.legendre.leggauss(64)
    t = 0.25 * math.pi * (xg + 1.0)                     # theta in (0, pi/2)
    wt = 0.25 * math.pi * wg
    s = np.sin(t)
    nuB = EE * B / (2.0 * math.pi * ME * CL)
    nuc = (2.0 / 9.0) * nuB * th * th
    K2 = 2.0 * th * th if k2_mode == 1 else special.kv(2, 1.0 / th)
    A = math.sqrt(2.0) * math.pi * EE * EE * ne / (3.0 * CL * K2)
    X = (nu[:, None] / nuc) / s[None, :]
    G = (np.sqrt(X) + 2.0 ** (11.0 / 12.0) * np.cbrt(np.sqrt(X))) ** 2 * np.exp(-np.cbrt(X))
    F = (s * s * G * wt).sum(axis=1)
    return 4.0 * math.pi * A * nuc * F


@pytest.mark.parametrize("a,R_high", [(0.9375, 20.0), (-0.94, 1.0)])   # the retrograde torus is cooler
def test_birth_weights_and_power_on_a_torus(oracle_mod, a, R_high):
    p, g = synth.torus(a=a, n1=48, n2=24, seed=11, scatter=0, R_high=R_high)
    p = dict(p, w_min=1e-300)   # the table without its floor: the identities hold for any table
    M = oracle_mod.Model(p, g)
    tot = M.prepare(3e5, 9)
    X, K, w = M.emit()
    # a frequency drawn past the emissivity table's end (where j_nu = 0 but g_lin > 0) carries w = 0
    assert len(w) == tot > 10000 and np.all(w >= 0) and (w > 0).mean() > 0.99
    # zone centres, volumes sqrt(-g) d^3x L^3 with sqrt(-g) = Sigma sin(theta) r dtheta/dx2 (x1 = ln r)
    n1, n2, n3 = g["n1"], g["n2"], g["n3"]
    i, j, k = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    x1 = g["x1_0"] + (i.ravel() + 0.5) * g["dx1"]
    x2 = g["x2_0"] + (j.ravel() + 0.5) * g["dx2"]
    x3 = g["x3_0"] + (k.ravel() + 0.5) * g["dx3"]
    h = p["hslope"]
    r = np.exp(x1)
    th = math.pi * x2 + 0.5 * (1.0 - h) * np.sin(2.0 * math.pi * x2)
    dth = math.pi * (1.0 + (1.0 - h) * np.cos(2.0 * math.pi * x2))
    sig = r * r + a * a * np.cos(th) ** 2
    vol = sig * np.sin(th) * r * dth * g["dx1"] * g["dx2"] * g["dx3"] * p["L_unit"] ** 3
    assert vol == pytest.approx(M.zones()["vol"], rel=1e-12)
    lnu = np.linspace(math.log(p["nu_min"]), math.log(p["nu_max"]), 401)   # trapezoid error ~1e-5
    nu = np.exp(lnu)
    n_phot, power = 0.0, 0.0
    for q in range(len(x1)):
        f = M.fluid(np.array([0.0, x1[q], x2[q], x3[q]]))
        if not (f["plasma"] and f["thetae"] >= p["thetae_min"] and f["ne"] > 0 and f["B"] > 0):
            continue
        jn = angle_integrated_jnu(nu, f["ne"], f["thetae"], f["B"], p.get("k2_mode", 0))
        n_phot += vol[q] / HPL * np.trapezoid(jn, lnu)
        power += vol[q] * np.trapezoid(jn * nu, lnu)
    # superphotons are born at their zone's centre: fluid-frame energy of each birth wavevector,
    # -k.u with the metric and 4-velocity of that centre (h nu = eps m_e c^2)
    zone = (np.floor((X[:, 1] - g["x1_0"]) / g["dx1"]).astype(int) * n2
            + np.floor((X[:, 2] - g["x2_0"]) / g["dx2"]).astype(int)) * n3 \
        + np.floor((X[:, 3] - g["x3_0"]) / g["dx3"]).astype(int)
    ucov = np.zeros((len(x1), 4))
    for q in np.unique(zone):
        Xc = np.array([0.0, x1[q], x2[q], x3[q]])
        ucov[q] = oracle_mod.gcov(p, Xc) @ M.fluid(Xc)["ucon"]
    assert np.allclose(X[:, 1], x1[zone]) and np.allclose(X[:, 2], x2[zone])
    eps = -(K * ucov[zone]).sum(axis=1)
    nu_f = eps * ME * CL * CL / HPL
    assert np.all((nu_f > 0.99 * p["nu_min"]) & (nu_f < 1.01 * p["nu_max"]))
    # Monte Carlo error of the sums: the counts are stratified by zone (floor(n_i) or floor(n_i) + 1),
    # so the variance is the within-zone spread of the weights plus the rounding of each count
    nbar = M.zones()["nbar"]
    frac = nbar - np.floor(nbar)

    def sigma(v):
        cnt = np.bincount(zone, minlength=len(nbar))
        s = np.bincount(zone, weights=v, minlength=len(nbar))
        s2 = np.bincount(zone, weights=v * v, minlength=len(nbar))
        m = np.where(cnt > 0, s / np.maximum(cnt, 1), 0.0)
        within = np.where(cnt > 1, s2 - cnt * m * m, 0.0)
        return math.sqrt(within.sum() + (frac * (1.0 - frac) * m * m).sum())

    v1, v2 = w, w * HPL * nu_f
    s1, s2 = v1.sum(), v2.sum()
    e1, e2 = sigma(v1), sigma(v2)
    assert e1 < 0.01 * s1 and e2 < 0.01 * s2   # the pins resolve departures of a few percent
    assert abs(s1 - n_phot) < 4.0 * e1 + 1e-3 * n_phot, (s1, n_phot, e1)
    assert abs(s2 - power) < 4.0 * e2 + 1e-3 * power, (s2, power, e2)
