"""The GRMHD-like workloads at their full sizes in their named forms, checked through properties
that hold at any size (the oracle cannot build the weights of a 4.7-million-zone turbulent grid
in test time; its parity with the device is tested on the same workloads at small sizes):
  - 2-D torus (a = 0.9375, 256 x 128, N_s = 1e7) with the coefficient surrogate;
  - 3-D snapshot (a = 0.5, 288 x 128 x 128 FP32, N_s = 1e8, 6 inclination bins) in mixed precision
    with the surrogate, and in the configuration's stated form: the split precision (FP64 geodesic,
    FP32 rest) with the surrogate.
Each named form's spectrum agrees with the plain FP64 run of the same job (FP64 itself is parity-
tested against the oracle) within 1 % in total luminosity and max(1 %, 3 sigma) per bin."""
import numpy as np
import pytest

from helpers import requires_gpu
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.fixture(scope="module")
def weights():
    from paper_2602_13198_gb300 import build, mc
    build.build()
    p, _ = synth.torus(n1=32, n2=16)
    m = mc.Model(p, precision="mixed")
    m.surrogate_train(n_train=1 << 18, steps=40000, batch=4096, lr=2e-3, seed=1)
    return m.surrogate_weights()


def run(p, g, n_s, seed, precision, w=None):
    from paper_2602_13198_gb300 import mc
    m = mc.Model(p, precision=precision, surrogate=w is not None)
    if w is not None:
        m.surrogate_weights(w)
    m.set_grid(g)
    st = m.run(n_s, seed)
    s = m.spectrum_sums().copy()
    del m
    return st, s


def compare(st_ref, s_ref, st, s, n_s):
    assert st["n_total"] == st_ref["n_total"] and st["n_emit"] == st_ref["n_emit"]
    # the expected total is N_s without the weight floor; the floor w_min only lowers it
    assert 0 < st["n_total"] <= n_s + 5.0 * np.sqrt(n_s)
    assert st["err_flags"] == 0 and st_ref["err_flags"] == 0
    lum_ref, lum = s_ref[..., 0].sum(), s[..., 0].sum()
    assert abs(lum / lum_ref - 1.0) < 0.01, (lum, lum_ref)
    a, b = s[..., 0], s_ref[..., 0]
    sig = np.sqrt(s[..., 1] + s_ref[..., 1])
    sel = (s[..., 2] >= 16) & (s_ref[..., 2] >= 16)
    bad = sel & (np.abs(a - b) > np.maximum(0.01 * np.abs(b), 3.0 * sig))
    # family-wise: a few 3-sigma excursions among hundreds of bins are expected
    assert bad.sum() <= max(2, 0.01 * sel.sum()), np.argwhere(bad)
    return abs(lum / lum_ref - 1.0)


def test_torus_2d_full_size_with_surrogate(weights):
    p, g = synth.torus()
    st0, s0 = run(p, g, 1e7, 1, "fp64")
    st1, s1 = run(p, g, 1e7, 1, "mixed", weights)
    e = compare(st0, s0, st1, s1, 1e7)
    print("2-D torus, surrogate vs FP64: total luminosity %.2e, %d superphotons" % (e, st1["n_emit"] + st1["n_child"]))


def test_snapshot_3d_full_size_mixed_and_split_with_surrogate(weights):
    p, g = synth.torus3d()
    assert (g["n1"], g["n2"], g["n3"]) == (288, 128, 128) and g["prim"].dtype == np.float32 and p["n_incl"] == 6
    st0, s0 = run(p, g, 1e8, 1, "fp64")
    for form in ("mixed", "split"):
        st1, s1 = run(p, g, 1e8, 1, form, weights)
        assert s1.shape[0] == 6
        e = compare(st0, s0, st1, s1, 1e8)
        print("3-D snapshot, %s + surrogate vs FP64: total luminosity %.2e, %d superphotons"
              % (form, e, st1["n_emit"] + st1["n_child"]))


def test_snapshot_3d_full_size_sampled_against_oracle():
    """The benchmark's main workload in its launch configuration (3-D snapshot, N_s = 1e8, shard 0 of 8,
    plain FP64) against the oracle: zone counts bit-exact over all 4.7 M zones, the shard's primaries
    the same, and per-superphoton end states of 400 sampled uids of the shard within 1e-9 (the oracle
    traces them one by one)."""
    from helpers import compare_logs, oracle_model
    from paper_2602_13198_gb300 import mc
    p, g = synth.torus3d()
    m = mc.Model(p, precision="fp64")
    m.set_grid(g)
    st = m.run(1e8, 1, shard=0, n_shards=8)
    om = oracle_model(p, dict(g, prim=np.asarray(g["prim"], dtype=np.float64)))
    tot = om.prepare(1e8, 1)
    assert st["n_total"] == tot
    assert np.array_equal(m.zone_counts(), om.zones()["counts"])
    u0, u1 = mc.shard_bounds(tot, 0, 8)
    assert st["n_emit"] == u1 - u0
    rng = np.random.default_rng(11)
    uids = np.sort(rng.choice(np.arange(u0, u1), size=400, replace=False))
    r = compare_logs(m.trace(1e8, 1, uids), om.run(uids=uids, log=True)["log"])
    assert r["n"] >= 0.99 * len(uids)
    assert len(r["flips"]) <= 2
    assert r["worst"]["X"] < 1e-9 and r["worst"]["K"] < 1e-9 and r["worst"]["w"] < 1e-7, r["worst"]

