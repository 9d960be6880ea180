"""The split precision form (MC_PREC_SPLIT): FP64 geodesic and step size; FP32 plasma coefficients,
optical depths, weights (relative to each superphoton's FP64 birth weight), scattering decision and
Compton kinematics.  Against the FP64 oracle through the C ABI:
- without scattering, positions and wavevectors follow the FP64 geodesic: traced end states within
  1e-9 in X and K (the geodesic arithmetic is the FP64 form's), weights of recorded superphotons
  within FP32 accumulation error;
- with scattering, zone counts bit-exact and every spectrum bin within max(1%, 3 sigma), on the
  scattering sphere, a Kerr torus (prograde and retrograde), a 3-D FP32 turbulent grid, and with
  kappa electrons and bremsstrahlung;
- the batched form equals each model's own split-form run, and the surrogate on the split form keeps
  the spectra within max(1%, 3 sigma) of the oracle."""
import numpy as np
import pytest

from helpers import compare_logs, gpu_model, oracle_model, requires_gpu, spectra_agree
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]


def test_split_form_is_accepted_and_checked():
    from paper_2602_13198_gb300 import mc
    p, _ = synth.sphere("flat", n1=4, n2=4)
    mc.Model(p, precision="split")
    with pytest.raises(mc.MCError):
        mc.Model(p, precision=3)


@pytest.mark.parametrize("kind,n_s,seed", [("ks_sphere", 1e5, 71), ("kerr_torus", 3e4, 72), ("retro_torus", 3e4, 73)])
def test_split_geodesics_match_fp64_oracle(kind, n_s, seed):
    if kind == "ks_sphere":
        p, g = synth.sphere("ks")
    elif kind == "kerr_torus":
        p, g = synth.torus(seed=7, a=0.9375, n1=96, n2=48, scatter=0)
    else:
        p, g = synth.torus(seed=8, a=-0.94, n1=96, n2=48, R_high=10.0, scatter=0)
    assert not p["scatter"]
    gm = gpu_model(p, g, precision="split")
    om = oracle_model(p, g)
    tot = om.prepare(n_s, seed)
    rng = np.random.default_rng(seed)
    uids = np.sort(rng.choice(tot, size=min(400, tot), replace=False))
    lg, lo = gm.trace(n_s, seed, uids), om.run(uids=uids, log=True)["log"]
    r = compare_logs(lg, lo)
    assert r["n"] >= 0.99 * len(uids)
    assert len(r["flips"]) <= max(2, 0.01 * r["n"]), len(r["flips"])
    assert r["worst"]["X"] < 1e-9 and r["worst"]["K"] < 1e-9, r["worst"]
    rec = compare_logs([x for x in lg if x["status"] == 1], [x for x in lo if x["status"] == 1])
    assert rec["n"] > 0 and rec["worst"]["w"] < 1e-3, rec["worst"]


def _cases():
    return {
        "ks_scatter": (synth.scattering_sphere(1e-1, n1=256, n2=64), 2e4, 81),
        "torus": (synth.torus(n1=64, n2=32), 2e4, 82),
        "retro_torus": (synth.torus(a=-0.5, n1=96, n2=48, R_high=1.0, M_unit=1e18, seed=61), 3e4, 83),
        "torus3d": (synth.torus3d(n1=48, n2=24, n3=16), 2e4, 84),
        "kappa": (synth.scattering_sphere(0.1, n1=256, n2=64, kappa=5.0), 2e4, 85),
        "brems": ((lambda pg: (dict(pg[0], brems=1), pg[1]))(synth.scattering_sphere(1e-1, n1=64, n2=16)), 1e4, 86),
    }


@pytest.mark.parametrize("name", ["ks_scatter", "torus", "retro_torus", "torus3d", "kappa", "brems"])
def test_split_spectra_match_oracle(name):
    (p, g), n_s, seed = _cases()[name]
    go = dict(g, prim=np.asarray(g["prim"], dtype=np.float64))
    gm = gpu_model(p, g, precision="split")
    st = gm.run(n_s, seed)
    om = oracle_model(p, go)
    tot = om.prepare(n_s, seed)
    assert st["n_total"] == tot
    assert np.array_equal(gm.zone_counts(), om.zones()["counts"])
    ro = om.run()
    ok, bad = spectra_agree(gm.spectrum_sums(), ro["spec"])
    assert ok, bad
    assert st["n_child"] > 0
    # scattered superphotons: the same number within a few (decisions taken in FP32 may flip near a
    # threshold), and the same total luminosity within 1%
    assert abs(st["n_child"] - ro["stats"]["n_child"]) <= max(3, 0.01 * ro["stats"]["n_child"])
    lg, lo = gm.spectrum_sums()[..., 0].sum(), ro["spec"][..., 0].sum()
    assert abs(lg - lo) <= 0.01 * lo


def test_split_batch_matches_individual_runs():
    from paper_2602_13198_gb300 import mc
    specs = [dict(a=0.94, n1=64, n2=32, R_high=10.0), dict(a=-0.5, n1=48, n2=24, R_high=1.0),
             dict(a=0.0, n1=96, n2=48, R_high=1.0)]
    models = [synth.torus(seed=300 + i, **kw) for i, kw in enumerate(specs)]
    ns = [3e4, 1e4, 2e4]
    seeds = [91, 92, 93]
    ref = []
    for (p, g), n_s, sd in zip(models, ns, seeds):
        m = mc.Model(p, precision="split")
        m.set_grid(g)
        ref.append((m.run(n_s, sd), m.spectrum_sums().copy()))
    ctxs = []
    for p, g in models:
        m = mc.Model(p, precision="split")
        m.set_grid(g)
        ctxs.append(m)
    for rep in range(2):
        st = mc.run_batch(ctxs, ns, seeds, autotune=(rep == 0), graph=True)
        assert st["n_emit"] == sum(r[0]["n_emit"] for r in ref)
        assert st["n_child"] == sum(r[0]["n_child"] for r in ref)
        for m, (rs, rspec) in zip(ctxs, ref):
            s = m.spectrum_sums()
            assert np.array_equal(s[..., 2], rspec[..., 2])
            assert np.allclose(s[..., :2], rspec[..., :2], rtol=1e-11, atol=0)


def test_split_with_surrogate_matches_oracle():
    from paper_2602_13198_gb300 import mc
    p0, _ = synth.sphere("flat", n1=4, n2=4)
    trainer = mc.Model(p0, precision="mixed")
    trainer.surrogate_train(n_train=1 << 17, steps=20000, batch=4096, lr=2e-3, seed=2)
    w = trainer.surrogate_weights()
    for (p, g), n_s, seed in (_cases()["ks_scatter"], _cases()["torus"]):
        m = mc.Model(p, precision="split", surrogate=True)
        m.surrogate_weights(w)
        m.set_grid(g)
        st = m.run(n_s, seed)
        om = oracle_model(p, g)
        assert om.prepare(n_s, seed) == st["n_total"]
        ok, bad = spectra_agree(m.spectrum_sums(), om.run()["spec"])
        assert ok, bad
