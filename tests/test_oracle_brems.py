"""Oracle pins of the thermal bremsstrahlung (future work in section 6; Stepney & Guilbert fits in the
form of Narayan & Yi 1995, flat Gaunt shape, Kirchhoff absorption): the two branches of each fit
meet at Theta_e = 1, the non-relativistic rate is the classical 1.4e-27 T^1/2 n_e n_i g_B with a
Gaunt factor in the usual range, the spectrum integrates to the rate, alpha_nu B_nu = j_nu, and a
bremsstrahlung-only thin sphere reproduces nu V 4 pi j_nu bin by bin."""
import math

import numpy as np
from scipy import integrate

from paper_2602_13198_gb300 import synth

ME, CL, KB, HPL = 9.1093837015e-28, 2.99792458e10, 1.380649e-16, 6.62607015e-27


def test_fits_are_continuous_at_theta_one():
    import oracle
    lo, hi = oracle.brems_q(1e10, 1.0 - 1e-12), oracle.brems_q(1e10, 1.0 + 1e-12)
    assert abs(hi / lo - 1.0) < 3e-3
    # and scale as n_e^2
    assert abs(oracle.brems_q(2e10, 0.3) / oracle.brems_q(1e10, 0.3) - 4.0) < 1e-12


def test_nonrelativistic_rate_is_classical():
    import oracle
    for T in (1e5, 1e6, 1e7):
        th = KB * T / (ME * CL * CL)
        gB = oracle.brems_q(1.0, th) / (1.4e-27 * math.sqrt(T))
        assert 1.1 < gB < 1.6, (T, gB)


def test_spectrum_integrates_to_the_rate_and_obeys_kirchhoff():
    import oracle
    p, _ = synth.sphere("flat", R=1.0, B_gauss=0.0, brems=1)
    for th in (0.05, 3.0):
        q = oracle.brems_q(1e13, th)
        nut = th * ME * CL * CL / HPL
        tot = integrate.quad(lambda x: oracle.brems_angint(p, x * nut, 1e13, th) * nut, 0, 60, epsabs=0, epsrel=1e-12)[0]
        assert abs(tot / q - 1.0) < 1e-9
        for nu in (1e9, 0.3 * nut, 3.0 * nut):
            j = oracle.brems_angint(p, nu, 1e13, th) / (4 * math.pi)
            bnu = oracle.bnu(nu, th)
            assert abs(oracle.brems_nu_alpha(p, nu, 1e13, th) * bnu / nu / j - 1.0) < 1e-12


def test_brems_only_thin_sphere_spectrum():
    import oracle
    th = 0.01
    p, g = synth.sphere("flat", R=1.0, ne=1e13, thetae=th, B_gauss=0.0, n1=128, n2=32, r_record=3000.0, brems=1)
    m = oracle.Model(p, g)
    m.prepare(4e4, 3)
    out = m.run(nthreads=16)
    st = out["stats"]
    assert st["n_emit"] > 0 and st["n_abs"] == 0
    dlog = (p["lnu_hi"] - p["lnu_lo"]) / p["n_bins"]
    dln = dlog * math.log(10)
    S = out["spec"][0]
    nuL, sig = S[:, 0] * ME * CL * CL / dln, np.sqrt(S[:, 1]) * ME * CL * CL / dln
    V = 4 * math.pi / 3 * (1 - math.exp(3 * g["x1_0"]))
    edges = p["lnu_lo"] + dlog * np.arange(p["n_bins"] + 1)
    nu_lo, nu_hi = math.log10(p["nu_min"]), math.log10(p["nu_max"])
    ref = np.array([integrate.quad(lambda l: 10 ** l * V * oracle.brems_angint(p, 10 ** l, 1e13, th),
                                   max(edges[i], nu_lo), min(edges[i + 1], nu_hi), epsrel=1e-10)[0] / dlog
                    if edges[i + 1] > nu_lo and edges[i] < nu_hi else 0.0 for i in range(p["n_bins"])])
    sel = S[:, 2] >= 200
    assert sel.sum() > 60
    z = (nuL[sel] - ref[sel]) / sig[sel]
    rel = np.abs(nuL[sel] / ref[sel] - 1.0)
    assert np.all((rel < 0.01) | (np.abs(z) < 4.0))
    assert abs(np.mean(z)) < 3.0 / math.sqrt(sel.sum())
