"""Per-generation bias tuning on the device: the same scales, counts and spectrum as the oracle's
tuned run of the same job, a trace after the run following the oracle photon by photon, and the
batched path refusing it."""
import numpy as np
import pytest

from helpers import compare_logs, gpu_model, oracle_model, requires_gpu, spectra_agree
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]


def case(target):
    p, g = synth.scattering_sphere(1e-1, n1=64, n2=16)
    return dict(p, bias_target=target), g


def test_tuned_run_matches_oracle():
    p, g = case(1.0)
    n_s, seed = 2e4, 9
    gm = gpu_model(p, g)
    st = gm.run(n_s, seed)
    om = oracle_model(p, g)
    tot = om.prepare(n_s, seed)
    ro = om.run(nthreads=8)
    assert st["n_total"] == tot
    assert np.allclose(gm.bias_scales(), om.bias_scales(), rtol=1e-12)
    assert gm.bias_scales()[1] > 1.0
    for k in ("n_emit", "n_child", "n_events"):
        assert abs(st[k] - ro["stats"][k]) <= max(2, 0.002 * ro["stats"][k]), k
    ok, bad = spectra_agree(gm.spectrum_sums(), ro["spec"])
    assert ok, bad
    # a trace after the run scatters with the run's scales: per-superphoton parity with the oracle
    uids = np.arange(0, tot, max(1, tot // 300))
    r = compare_logs(gm.trace(n_s, seed, uids), om.run(uids=uids, log=True)["log"])
    assert r["n"] >= 0.99 * len(uids) and len(r["flips"]) <= 2
    assert r["worst"]["X"] < 1e-9 and r["worst"]["K"] < 1e-9 and r["worst"]["w"] < 1e-7


def test_batched_run_refuses_tuning():
    from paper_2602_13198_gb300 import mc
    p, g = case(1.0)
    m = gpu_model(p, g)
    with pytest.raises(mc.MCError) as e:
        mc.run_batch([m], [1e3], [1], autotune=False, graph=False)
    assert e.value.code == -1
