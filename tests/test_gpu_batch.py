"""Batched survey: several models in one persistent cooperative launch (mc_run_batch) must give each
model exactly its individual mc_run result (superphoton streams are keyed per model uid), with and
without CUDA-graph capture and autotuning, in the plain, mixed and surrogate forms."""
import numpy as np
import pytest

from helpers import requires_gpu
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]


def survey_models(n=5):
    out = []
    specs = [dict(a=0.94, n1=64, n2=32, R_high=10.0), dict(a=-0.5, n1=48, n2=24, R_high=40.0),
             dict(a=0.0, n1=96, n2=48, R_high=1.0), dict(a=0.5, n1=40, n2=16, R_high=160.0, M_unit=2e18),
             dict(a=0.9375, n1=64, n2=32, R_high=20.0, M_unit=1e18)]
    for i, kw in enumerate(specs[:n]):
        p, g = synth.torus(seed=100 + i, **kw)
        out.append((p, g))
    return out


def individual(models, ns, seeds, precision, weights=None):
    from paper_2602_13198_gb300 import mc
    res = []
    for (p, g), n_s, sd in zip(models, ns, seeds):
        m = mc.Model(p, precision=precision, surrogate=weights is not None)
        if weights is not None:
            m.surrogate_weights(weights)
        m.set_grid(g)
        st = m.run(n_s, sd)
        res.append((st, m.spectrum_sums().copy()))
    return res


@pytest.mark.parametrize("precision,graph,autotune", [("fp64", False, False), ("mixed", True, True)])
def test_batch_matches_individual_runs(precision, graph, autotune):
    from paper_2602_13198_gb300 import build, mc
    build.build()
    models = survey_models()
    ns = [3e4, 1e4, 2e4, 5e3, 4e4]
    seeds = [11, 12, 13, 14, 15]
    ref = individual(models, ns, seeds, precision)
    ctxs = []
    for p, g in models:
        m = mc.Model(p, precision=precision)
        m.set_grid(g)
        ctxs.append(m)
    for rep in range(2):            # the second call replays the captured graph
        st = mc.run_batch(ctxs, ns, seeds, autotune=autotune, graph=graph)
        assert st["n_emit"] == sum(r[0]["n_emit"] for r in ref)
        assert st["n_child"] == sum(r[0]["n_child"] for r in ref)
        for m, (rs, rspec) in zip(ctxs, ref):
            s = m.spectrum_sums()
            assert np.array_equal(s[..., 2], rspec[..., 2])
            assert np.allclose(s[..., :2], rspec[..., :2], rtol=1e-11, atol=0)
        if graph:
            assert st["batch_graph"] == 1 or rep == 0


def test_batch_with_surrogate_matches_individual_runs():
    from paper_2602_13198_gb300 import mc
    p0, _ = synth.sphere("flat", n1=4, n2=4)
    trainer = mc.Model(p0, precision="mixed")
    trainer.surrogate_train(n_train=1 << 17, steps=20000, batch=4096, lr=2e-3, seed=2)
    w = trainer.surrogate_weights()
    models = survey_models(3)
    ns = [2e4, 1e4, 2e4]
    seeds = [21, 22, 23]
    ref = individual(models, ns, seeds, "mixed", weights=w)
    ctxs = []
    for p, g in models:
        m = mc.Model(p, precision="mixed", surrogate=True)
        m.surrogate_weights(w)
        m.set_grid(g)
        ctxs.append(m)
    st = mc.run_batch(ctxs, ns, seeds, autotune=False, graph=True)
    assert st["n_emit"] == sum(r[0]["n_emit"] for r in ref)
    for m, (rs, rspec) in zip(ctxs, ref):
        s = m.spectrum_sums()
        assert np.array_equal(s[..., 2], rspec[..., 2])
        assert np.allclose(s[..., :2], rspec[..., :2], rtol=1e-11, atol=0)


def test_batch_rejects_mixed_modes():
    from paper_2602_13198_gb300 import mc
    models = survey_models(2)
    a = mc.Model(models[0][0], precision="fp64")
    a.set_grid(models[0][1])
    b = mc.Model(models[1][0], precision="mixed")
    b.set_grid(models[1][1])
    with pytest.raises(mc.MCError) as e:
        mc.run_batch([a, b], [1e3, 1e3], [1, 2])
    assert e.value.code == -1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_mixes_electron_models(precision):
    # thermal, kappa (emission, absorption and scattering) and bremsstrahlung models share one launch;
    # each model reads its own tables through its descriptor
    from paper_2602_13198_gb300 import mc
    models = [synth.torus(seed=201, a=0.5, n1=48, n2=24, kappa=4.0),
              synth.scattering_sphere(0.1, n1=128, n2=32, kappa=5.0),
              synth.torus(seed=202, a=0.0, n1=48, n2=24, brems=1),
              synth.torus(seed=203, a=0.9, n1=48, n2=24)]
    ns = [2e4, 1e4, 2e4, 1e4]
    seeds = [31, 32, 33, 34]
    ref = individual(models, ns, seeds, precision)
    ctxs = []
    for p, g in models:
        m = mc.Model(p, precision=precision)
        m.set_grid(g)
        ctxs.append(m)
    st = mc.run_batch(ctxs, ns, seeds, autotune=False, graph=False)
    assert st["n_emit"] == sum(r[0]["n_emit"] for r in ref)
    assert st["n_child"] == sum(r[0]["n_child"] for r in ref) and st["n_child"] > 0
    for m, (rs, rspec) in zip(ctxs, ref):
        s = m.spectrum_sums()
        assert np.array_equal(s[..., 2], rspec[..., 2])
        assert np.allclose(s[..., :2], rspec[..., :2], rtol=1e-11, atol=0)


def test_batch_barrier_wait_limit_times_out_and_context_recovers():
    # a 1 microsecond limit makes the first CTAs at the first grid barrier give up while every CTA is
    # still present: the launch must end with MC_ERR_TIMEOUT, and the same contexts must then run the
    # batch to the individual results once the default limit is back (direct launch and graph)
    from paper_2602_13198_gb300 import mc
    models = survey_models(3)
    ns = [2e4, 1e4, 2e4]
    seeds = [41, 42, 43]
    ref = individual(models, ns, seeds, "fp64")
    ctxs = []
    for p, g in models:
        m = mc.Model(p, precision="fp64")
        m.set_grid(g)
        ctxs.append(m)
    with pytest.raises(mc.MCError) as e:
        ctxs[0].set_wait_limit(0.0)
    assert e.value.code == -1
    for graph in (False, True):
        ctxs[0].set_wait_limit(1e-6)
        with pytest.raises(mc.MCError) as e:
            mc.run_batch(ctxs, ns, seeds, autotune=False, graph=graph)
        assert e.value.code == -4                  # MC_ERR_TIMEOUT
        ctxs[0].set_wait_limit(120.0)
        st = mc.run_batch(ctxs, ns, seeds, autotune=False, graph=graph)
        assert st["n_emit"] == sum(r[0]["n_emit"] for r in ref)
        for m, (rs, rspec) in zip(ctxs, ref):
            s = m.spectrum_sums()
            assert np.array_equal(s[..., 2], rspec[..., 2])
            assert np.allclose(s[..., :2], rspec[..., :2], rtol=1e-11, atol=0)
