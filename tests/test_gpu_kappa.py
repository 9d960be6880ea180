"""Kappa-electron synchrotron emission and absorption on the device against the oracle (independent
tables on the same grid): a thin flat sphere and the Schwarzschild sphere (absorbing below ~1e13 Hz)
with kappa = 4, FP64 and mixed precision; the surrogate refuses kappa."""
import numpy as np
import pytest

from helpers import compare_logs, gpu_model, oracle_model, requires_gpu, spectra_agree
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]


def cases():
    thin = synth.sphere("flat", R=1.0, ne=1e13, thetae=100.0, B_gauss=1.0, n1=128, n2=32, r_record=3000.0, kappa=4.0)
    ks = synth.sphere("ks", n1=256, n2=64, kappa=4.0)
    return {"flat_thin": thin, "ks_sphere": ks}


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
