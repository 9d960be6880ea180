"""Kappa-electron synchrotron emission and absorption on the device against the oracle (independent
tables on the same grid): a thin flat sphere and the Schwarzschild sphere (absorbing below ~1e13 Hz)
with kappa = 4, FP64 and mixed precision; the surrogate refuses kappa.  Compton scattering off the
kappa population (hot cross-section table and Lorentz-factor sampler): scattering spheres with
w = 1.6 (kappa = 5, Theta_e = 4) and w = 1/7 (kappa = 3.5, Theta_e = 1), the two envelopes of the sampler.
(An input with w = 1 exactly would let the last bit of each side's Theta_e pick the envelope, and the
two sides would then draw different, equally valid, electrons.)  The two codes integrate the kappa hot
cross-section with different rules (trapezoid in ln(gamma - 1) against Gauss-Legendre panels), and
sigma_KN's small-argument branch (1 - 2x below x = 1e-3) steps by ~5e-6 there, so the tables agree
to ~1e-8 rather than to rounding; event points and the children's paths inherit that, hence the
1e-7 bound on X and K in place of 1e-9."""
import numpy as np
import pytest

from helpers import compare_logs, gpu_model, oracle_model, requires_gpu, spectra_agree
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]


def cases():
    thin = synth.sphere("flat", R=1.0, ne=1e13, thetae=100.0, B_gauss=1.0, n1=128, n2=32, r_record=3000.0, kappa=4.0)
    ks = synth.sphere("ks", n1=256, n2=64, kappa=4.0)
    sc5 = synth.scattering_sphere(0.1, n1=256, n2=64, kappa=5.0)
    sc35 = synth.scattering_sphere(0.1, n1=256, n2=64, thetae=1.0, kappa=3.5)
    return {"flat_thin": thin, "ks_sphere": ks, "scatter_k5": sc5, "scatter_k35": sc35}


@pytest.mark.parametrize("name,n_s,seed", [("flat_thin", 2e4, 1), ("ks_sphere", 3e4, 2)])
def test_parity_with_oracle(name, n_s, seed):
    p, g = cases()[name]
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
    if name == "ks_sphere":
        assert st["n_abs"] > 0      # the low-frequency superphotons are absorbed


def test_mixed_precision_kappa():
    p, g = cases()["ks_sphere"]
    gm = gpu_model(p, g, precision="mixed")
    gm.run(3e4, 3)
    om = oracle_model(p, g)
    om.prepare(3e4, 3)
    ok, bad = spectra_agree(gm.spectrum_sums(), om.run(nthreads=8)["spec"])
    assert ok, bad


def test_surrogate_refuses_kappa():
    from paper_2602_13198_gb300 import mc
    p, _ = cases()["flat_thin"]
    with pytest.raises(mc.MCError) as e:
        mc.Model(p, precision="mixed", surrogate=True)
    assert e.value.code == -1


@pytest.mark.parametrize("name,n_s,seed", [("scatter_k5", 2e4, 4), ("scatter_k35", 2e4, 5)])
def test_scattering_parity_with_oracle(name, n_s, seed):
    p, g = cases()[name]
    gm = gpu_model(p, g)
    st = gm.run(n_s, seed)
    om = oracle_model(p, g)
    tot = om.prepare(n_s, seed)
    assert st["n_total"] == tot
    ro = om.run(nthreads=8)
    assert st["n_child"] > 0
    for k in ("n_emit", "n_child", "n_rec", "n_capt"):
        assert abs(st[k] - ro["stats"][k]) <= max(2, 2e-3 * ro["stats"][k]), k
    ok, bad = spectra_agree(gm.spectrum_sums(), ro["spec"])
    assert ok, bad
    rng = np.random.default_rng(seed)
    uids = np.sort(rng.choice(tot, size=min(600, tot), replace=False))
    r = compare_logs(gm.trace(n_s, seed, uids), om.run(uids=uids, log=True)["log"])
    assert r["n"] >= 0.99 * len(uids) and len(r["flips"]) <= max(1, 0.002 * r["n"])
    assert r["worst"]["X"] < 1e-7 and r["worst"]["K"] < 1e-7 and r["worst"]["w"] < 1e-7


def test_scattering_mixed_precision_kappa():
    p, g = cases()["scatter_k5"]
    gm = gpu_model(p, g, precision="mixed")
    gm.run(2e4, 6)
    om = oracle_model(p, g)
    om.prepare(2e4, 6)
    ok, bad = spectra_agree(gm.spectrum_sums(), om.run(nthreads=8)["spec"])
    assert ok, bad
