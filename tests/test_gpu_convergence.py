"""Convergence study of the optically thin flat sphere on the GPU (section 4.1): R = 1 cm inside a
grid to r_out = 1e4 cm, Theta_e = 100, n_e = 1e13, B = 1 G, record at 3000 cm.  The normalised
integrated error eps_err (eq. conv_parameter) against the analytic nu (4 pi R^3 / 3) int dOmega j_nu
(eq. Lnu_analytic_thin_test) falls as N_s^-1/2 from 1e4 to 1e7 superphotons on 8192 radial cells.
At N_s = 1e8 the paper moves to 32000 radial cells with 5 x 5 partial cells at the sphere edge;
there the error stays on the N_s^-1/2 line and every well-populated bin is within 1 %, while the
abrupt edge (zone centre decides) of 8192 cells carries a volume bias that shows in eps_err."""
import math

import numpy as np
import pytest
from scipy import integrate

from helpers import requires_gpu
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]

ME, CL = 9.1093837015e-28, 2.99792458e10


def case(n1, partial):
    return synth.sphere("flat", R=1.0, ne=1e13, thetae=100.0, B_gauss=1.0, n1=n1, n2=128, r_record=3000.0,
                        r_out=1e4, partial=partial)


def nuLnu(p, sums):
    dln = (p["lnu_hi"] - p["lnu_lo"]) / p["n_bins"] * math.log(10)
    S = sums[0]
    return S[:, 0] * ME * CL * CL / dln, S[:, 2]


@pytest.fixture(scope="module")
def reference():
    import oracle
    p, _ = case(64, 0)
    dlog = (p["lnu_hi"] - p["lnu_lo"]) / p["n_bins"]
    edges = p["lnu_lo"] + dlog * np.arange(p["n_bins"] + 1)
    V = 4.0 * math.pi / 3.0

    def f(l):
        nu = 10.0 ** l
        return nu * V * oracle.jnu_angint(p, nu, 1e13, 100.0, 1.0)
    ref = np.array([integrate.quad(f, edges[i], edges[i + 1], epsrel=1e-10)[0] / dlog for i in range(p["n_bins"])])
    lg = 0.5 * (edges[1:] + edges[:-1])
    band = (lg > 8.5) & (lg < 14.0)
    return ref, band


def eps_err(nuL, ref, band):
    # (1 / Delta log nu) int |L_ref - L| / L_ref d log nu over the band of uniform log bins
    return float(np.mean(np.abs(ref[band] - nuL[band]) / ref[band]))


def run(n1, partial, n_s, seed):
    from helpers import gpu_model
    p, g = case(n1, partial)
    m = gpu_model(p, g)
    st = m.run(n_s, seed)
    assert st["n_abs"] == 0 and st["n_maxst"] == 0 and st["n_rec"] == st["n_emit"]
    return p, m.spectrum_sums()


def test_convergence_and_partial_cells(reference):
    ref, band = reference
    ns_list = [1e4, 1e5, 1e6, 1e7]
    errs = []
    for k, ns in enumerate(ns_list):
        p, s = run(8192, 0, ns, 11 + k)
        errs.append(eps_err(nuLnu(p, s)[0], ref, band))
    slope = np.polyfit(np.log10(ns_list), np.log10(errs), 1)[0]
    p, s_part = run(32000, 5, 1e8, 21)
    nuL, cnt = nuLnu(p, s_part)
    e_part = eps_err(nuL, ref, band)
    p, s_abr = run(8192, 0, 1e8, 22)
    e_abr = eps_err(nuLnu(p, s_abr)[0], ref, band)
    bias = lambda s_: float(np.mean(nuLnu(p, s_)[0][band] / ref[band] - 1.0))
    print("eps_err 1e4..1e7 (8192 cells): %s  slope %.3f; 1e8: partial cells (32000) %.2e (mean dev %.1e), "
          "abrupt (8192) %.2e (mean dev %.1e)" % (["%.2e" % e for e in errs], slope, e_part, bias(s_part), e_abr,
                                                  bias(s_abr)))
    assert abs(slope + 0.5) < 0.08
    # N_s = 1e8 with partial cells stays on the N_s^-1/2 line through the 1e4..1e7 points
    line = 10 ** np.polyval(np.polyfit(np.log10(ns_list), np.log10(errs), 1), 8.0)
    assert e_part < 1.3 * line
    # the abrupt edge's volume bias (~9e-4) adds to the ~7e-4 Monte Carlo error
    assert e_abr > e_part
    # every bin with >= 1e4 superphotons within 1 % of the analytic spectrum (the paper's figure)
    sel = band & (cnt >= 1e4)
    assert sel.sum() > 40
    assert np.all(np.abs(nuL[sel] / ref[sel] - 1.0) < 0.01)
