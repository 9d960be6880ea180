"""Thermal bremsstrahlung on the device against the oracle: a bremsstrahlung-only thin sphere
(no field: isotropic emission in the scattering tetrad's frame) and the scattering sphere with both
processes (the emitting process drawn per superphoton), FP64 and mixed precision; and the
bremsstrahlung-only spectrum against nu V 4 pi j_nu."""
import math

import numpy as np
import pytest
from scipy import integrate

from helpers import compare_logs, gpu_model, oracle_model, requires_gpu, spectra_agree
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]
ME, CL = 9.1093837015e-28, 2.99792458e10


def brems_sphere():
    return synth.sphere("flat", R=1.0, ne=1e13, thetae=0.01, B_gauss=0.0, n1=128, n2=32, r_record=3000.0, brems=1)


def both_sphere():
    p, g = synth.scattering_sphere(1e-1, n1=64, n2=16)
    return dict(p, brems=1), g


@pytest.mark.parametrize("name,n_s,seed", [("brems_only", 2e4, 1), ("synchrotron_and_brems", 1e4, 2)])
def test_parity_with_oracle(name, n_s, seed):
    p, g = brems_sphere() if name == "brems_only" else both_sphere()
    gm = gpu_model(p, g)
    st = gm.run(n_s, seed)
    om = oracle_model(p, g)
    tot = om.prepare(n_s, seed)
    assert st["n_total"] == tot
    assert np.array_equal(gm.zone_counts(), om.zones()["counts"])
    ro = om.run(nthreads=8)
    ok, bad = spectra_agree(gm.spectrum_sums(), ro["spec"])
    assert ok, bad
    uids = np.arange(0, tot, max(1, tot // 400))
    r = compare_logs(gm.trace(n_s, seed, uids), om.run(uids=uids, log=True)["log"])
    assert r["n"] >= 0.99 * len(uids) and len(r["flips"]) <= 2
    assert r["worst"]["X"] < 1e-9 and r["worst"]["K"] < 1e-9 and r["worst"]["w"] < 1e-7


def test_mixed_precision_with_brems():
    p, g = both_sphere()
    gm = gpu_model(p, g, precision="mixed")
    gm.run(1e4, 3)
    om = oracle_model(p, g)
    om.prepare(1e4, 3)
    ok, bad = spectra_agree(gm.spectrum_sums(), om.run(nthreads=8)["spec"])
    assert ok, bad


def test_brems_only_spectrum_vs_analytic():
    import oracle
    p, g = brems_sphere()
    gm = gpu_model(p, g)
    st = gm.run(1e6, 5)
    assert st["n_abs"] == 0
    S = gm.spectrum_sums()[0]
    dlog = (p["lnu_hi"] - p["lnu_lo"]) / p["n_bins"]
    dln = dlog * math.log(10)
    nuL, sig = S[:, 0] * ME * CL * CL / dln, np.sqrt(S[:, 1]) * ME * CL * CL / dln
    V = 4 * math.pi / 3 * (1 - math.exp(3 * g["x1_0"]))
    edges = p["lnu_lo"] + dlog * np.arange(p["n_bins"] + 1)
    lo, hi = math.log10(p["nu_min"]), math.log10(p["nu_max"])
    ref = np.zeros(p["n_bins"])
    for i in range(p["n_bins"]):
        a, b = max(edges[i], lo), min(edges[i + 1], hi)
        if b > a:
            ref[i] = integrate.quad(lambda l: 10 ** l * V * oracle.brems_angint(p, 10 ** l, 1e13, 0.01), a, b,
                                    epsrel=1e-10)[0] / dlog
    sel = S[:, 2] >= 2000
    assert sel.sum() > 60
    rel = nuL[sel] / ref[sel] - 1.0
    z = (nuL[sel] - ref[sel]) / sig[sel]
    assert np.all((np.abs(rel) < 0.01) | (np.abs(z) < 4.0))
    assert abs(np.mean(z)) < 3.0 / math.sqrt(sel.sum())


def test_surrogate_refuses_brems():
    from paper_2602_13198_gb300 import mc
    p, _ = both_sphere()
    with pytest.raises(mc.MCError) as e:
        mc.Model(p, precision="mixed", surrogate=True)
    assert e.value.code == -1
