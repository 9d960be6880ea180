"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded
inputs.  Zone counts bit-exact; per-superphoton FP64 end states within 1e-9 relative
(decision flips counted and bounded); spectra within max(1%, 3 Monte Carlo sigma)."""
import math

import numpy as np
import pytest

from helpers import compare_logs, flat_sphere, gpu_model, oracle_model, requires_gpu, spectra_agree
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]


def cases():
    out = {}
    out["flat_thin"] = flat_sphere()
    # Schwarzschild sphere of radius 10 GM/c^2 (n_e 1e13, Theta_e 10, B 10 G), full 1024 x 128 grid
    out["ks_sphere"] = synth.sphere("ks")
    # scattering sphere, tau_T = 0.1 (frequent scattering, bias clamps to 1)
    out["ks_scatter"] = synth.scattering_sphere(0.1, n1=256, n2=64)
    return out


@pytest.fixture(scope="module")
def case_data():
    return cases()


@pytest.mark.parametrize("name,n_s,seed", [("flat_thin", 3e4, 1), ("ks_sphere", 1e5, 1), ("ks_scatter", 2e4, 2)])
def test_zone_counts_bit_exact(case_data, name, n_s, seed):
    p, g = case_data[name]
    gm = gpu_model(p, g)
    st = gm.run(n_s, seed)
    om = oracle_model(p, g)
    tot = om.prepare(n_s, seed)
    assert st["n_total"] == tot
    assert np.array_equal(gm.zone_counts(), om.zones()["counts"])


@pytest.mark.parametrize("name,n_s,seed,nsample", [("flat_thin", 3e4, 1, 400), ("ks_sphere", 1e5, 1, 400),
                                                   ("ks_scatter", 2e4, 2, 600)])
def test_superphoton_end_states_fp64(case_data, name, n_s, seed, nsample):
    p, g = case_data[name]
    gm = gpu_model(p, g)
    om = oracle_model(p, g)
    tot = om.prepare(n_s, seed)
    rng = np.random.default_rng(seed)
    uids = np.sort(rng.choice(tot, size=min(nsample, tot), replace=False))
    lg = gm.trace(n_s, seed, uids)
    lo = om.run(uids=uids, log=True)["log"]
    r = compare_logs(lg, lo)
    assert r["n"] >= 0.99 * len(lo)
    assert len(r["flips"]) <= max(1, 0.002 * r["n"])
    assert r["worst"]["X"] < 1e-9 and r["worst"]["K"] < 1e-9
    assert r["worst"]["w"] < 1e-7


@pytest.mark.parametrize("name,n_s,seed", [("flat_thin", 2e4, 3), ("ks_scatter", 1e4, 4)])
def test_spectrum_fp64(case_data, name, n_s, seed):
    p, g = case_data[name]
    gm = gpu_model(p, g)
    stg = gm.run(n_s, seed)
    om = oracle_model(p, g)
    om.prepare(n_s, seed)
    ro = om.run()
    ok, bad = spectra_agree(gm.spectrum_sums(), ro["spec"])
    assert ok, bad
    so = ro["stats"]
    for k in ("n_emit", "n_child", "n_rec", "n_capt"):
        assert abs(stg[k] - so[k]) <= max(2, 2e-3 * so[k]), k


@pytest.mark.parametrize("name,n_s,seed", [("flat_thin", 2e4, 5), ("ks_scatter", 1e4, 6)])
def test_spectrum_mixed_precision(case_data, name, n_s, seed):
    p, g = case_data[name]
    gm = gpu_model(p, g, precision="mixed")
    gm.run(n_s, seed)
    om = oracle_model(p, g)
    om.prepare(n_s, seed)
    ro = om.run()
    ok, bad = spectra_agree(gm.spectrum_sums(), ro["spec"])
    assert ok, bad


def test_shards_sum_to_whole(case_data):
    p, g = case_data["ks_scatter"]
    gm = gpu_model(p, g)
    whole = gm.run(1e4, 9)
    s_whole = gm.spectrum_sums().copy()
    acc = np.zeros_like(s_whole)
    n_emit = 0
    for s in range(3):
        st = gm.run(1e4, 9, shard=s, n_shards=3)
        acc += gm.spectrum_sums()
        n_emit += st["n_emit"]
    assert n_emit == whole["n_emit"] == whole["n_total"]
    assert np.array_equal(acc[..., 2], s_whole[..., 2])
    assert np.allclose(acc[..., :2], s_whole[..., :2], rtol=1e-12, atol=0)


def test_run_is_deterministic_and_seeded(case_data):
    p, g = case_data["flat_thin"]
    gm = gpu_model(p, g)
    gm.run(5e3, 11)
    a = gm.spectrum_sums().copy()
    gm.run(5e3, 11)
    b = gm.spectrum_sums().copy()
    gm.run(5e3, 12)
    c = gm.spectrum_sums().copy()
    assert np.array_equal(a[..., 2], b[..., 2]) and np.allclose(a, b, rtol=1e-12, atol=0)
    assert not np.array_equal(a[..., 2], c[..., 2])


def test_edge_cases_and_errors():
    from paper_2602_13198_gb300 import mc
    p, g = flat_sphere(n1=2, n2=2)
    m = mc.Model(p)
    with pytest.raises(mc.MCError) as e:
        m.run(10, 1)
    assert e.value.code == -8          # STATE: no grid yet
    m.set_grid(g)
    st = m.run(0.01, 1)                # almost surely zero superphotons
    assert st["n_total"] == st["n_emit"] <= 1
    with pytest.raises(mc.MCError) as e:
        m.run(-1.0, 1)
    assert e.value.code == -1
    bad = dict(p, n_nu=1)
    with pytest.raises(mc.MCError):
        mc.Model(bad)
    g2 = dict(g)
    pr = g["prim"].copy()
    pr[0, 0] = np.nan
    g2["prim"] = pr
    with pytest.raises(mc.MCError) as e:
        m.set_grid(g2)
    assert e.value.code == -6          # NAN_INPUT


def test_queue_grows_when_a_generation_overflows():
    # optically thick torus (~30 scattered children per primary): the first scattered generation
    # outgrows the initial 2^20-slot queue, the run is redone with larger queues, and the result
    # equals a second run on the already-grown context (streams are keyed per superphoton)
    p, g = synth.torus(a=0.9375, n1=64, n2=32, R_high=20.0, M_unit=4e18, seed=104)
    gm = gpu_model(p, g)
    st1 = gm.run(5e5, 1)
    s1 = gm.spectrum_sums().copy()
    assert st1["n_child"] > (1 << 20)
    st2 = gm.run(5e5, 1)
    s2 = gm.spectrum_sums().copy()
    for k in ("n_total", "n_emit", "n_child", "n_rec", "n_abs", "n_capt", "n_steps", "n_events"):
        assert st1[k] == st2[k], k
    assert np.array_equal(s1[..., 2], s2[..., 2]) and np.allclose(s1, s2, rtol=1e-10, atol=0)


def test_ragged_3d_float32_grid():
    # 3-D grid with ragged sizes in FP32 storage (the layout of the 3-D snapshot workload)
    p, g = synth.sphere("ks", n1=37, n2=19, R=10.0)
    g3 = dict(g)
    n3 = 5
    pr = np.repeat(g["prim"].reshape(8, 37, 19, 1), n3, axis=3).reshape(8, -1)
    rng = np.random.default_rng(3)
    pr[0] *= np.exp(0.1 * rng.standard_normal(pr.shape[1]))
    g3.update(n3=n3, dx3=2 * math.pi / n3, prim=pr.astype(np.float32))
    go = dict(g3, prim=pr.astype(np.float32).astype(np.float64))
    gm = gpu_model(p, g3)
    st = gm.run(2e4, 5)
    om = oracle_model(p, go)
    tot = om.prepare(2e4, 5)
    assert st["n_total"] == tot
    assert np.array_equal(gm.zone_counts(), om.zones()["counts"])
    uids = np.arange(0, tot, max(1, tot // 300))
    r = compare_logs(gm.trace(2e4, 5, uids), om.run(uids=uids, log=True)["log"])
    assert len(r["flips"]) <= 1 and r["worst"]["X"] < 1e-9 and r["worst"]["K"] < 1e-9


# ------------------------------------------------------------------ GRMHD-like stand-ins (section 4.3)
@pytest.fixture(scope="module")
def tori():
    out = {}
    out["torus_small"] = synth.torus(n1=64, n2=32)
    out["torus3d_small"] = synth.torus3d(n1=48, n2=24, n3=16)
    return out


@pytest.mark.parametrize("name,n_s,seed", [("torus_small", 2e4, 1), ("torus3d_small", 2e4, 2)])
def test_torus_counts_end_states_and_spectrum(tori, name, n_s, seed):
    p, g = tori[name]
    go = dict(g, prim=np.asarray(g["prim"], dtype=np.float64))   # oracle reads the same (rounded) values
    gm = gpu_model(p, g)
    st = gm.run(n_s, seed)
    om = oracle_model(p, go)
    tot = om.prepare(n_s, seed)
    assert st["n_total"] == tot
    assert np.array_equal(gm.zone_counts(), om.zones()["counts"])
    ro = om.run(log=True)
    ok, bad = spectra_agree(gm.spectrum_sums(), ro["spec"])
    assert ok, bad
    uids = np.arange(0, tot, max(1, tot // 500))
    r = compare_logs(gm.trace(n_s, seed, uids), om.run(uids=uids, log=True)["log"])
    assert r["n"] >= 0.99 * len(uids)
    assert len(r["flips"]) <= max(1, 0.002 * r["n"])
    assert r["worst"]["X"] < 1e-9 and r["worst"]["K"] < 1e-9 and r["worst"]["w"] < 1e-7
    assert st["n_child"] > 0


def test_torus_full_size_sampled():
    # the 2-D GRMHD-like workload at its full size (256 x 128, N_s = 1e7): bit-exact counts, and
    # per-superphoton parity on a sample of uids the oracle can trace one by one
    p, g = synth.torus()
    gm = gpu_model(p, g)
    st = gm.run(1e7, 1)
    om = oracle_model(p, g)
    tot = om.prepare(1e7, 1)
    assert st["n_total"] == tot
    assert np.array_equal(gm.zone_counts(), om.zones()["counts"])
    rng = np.random.default_rng(7)
    uids = np.sort(rng.choice(tot, size=400, replace=False))
    r = compare_logs(gm.trace(1e7, 1, uids), om.run(uids=uids, log=True)["log"])
    assert r["n"] >= 0.99 * len(uids)
    assert len(r["flips"]) <= 2
    assert r["worst"]["X"] < 1e-9 and r["worst"]["K"] < 1e-9


def test_scattering_sphere_full_size_sampled():
    # the benchmark workload at full size (1024 x 128, N_s = 1e7), per-superphoton parity on samples
    p, g = synth.scattering_sphere(1e-1)
    gm = gpu_model(p, g)
    st = gm.run(1e7, 3)
    om = oracle_model(p, g)
    tot = om.prepare(1e7, 3)
    assert st["n_total"] == tot
    assert np.array_equal(gm.zone_counts(), om.zones()["counts"])
    rng = np.random.default_rng(8)
    uids = np.sort(rng.choice(tot, size=600, replace=False))
    r = compare_logs(gm.trace(1e7, 3, uids), om.run(uids=uids, log=True)["log"])
    assert r["n"] >= 0.99 * len(uids)
    assert len(r["flips"]) <= 2
    assert r["worst"]["X"] < 1e-9 and r["worst"]["K"] < 1e-9


@pytest.mark.parametrize("kind,n_s,seed", [("ks_sphere", 1e5, 21), ("kerr_torus", 3e4, 22)])
def test_mixed_precision_geodesics_match_fp64_oracle(kind, n_s, seed):
    # Without scattering, a superphoton's positions and wavevectors depend on the geodesic alone, so
    # the mixed form's double-float geodesic (48-bit significand, own e^x and sin/cos(pi x)) must
    # follow the oracle's FP64 paths closely; an FP32 geodesic would be off by ~1e-5.  Weights carry
    # the FP32 coefficients and are compared loosely.  The Kerr torus (a = 0.9375, h = 0.3)
    # exercises the spin terms and the theta map.
    if kind == "ks_sphere":
        p, g = synth.sphere("ks")
    else:
        p, g = synth.torus(seed=7, a=0.9375, n1=96, n2=48, scatter=0)
    assert not p["scatter"]
    gm = gpu_model(p, g, precision="mixed")
    om = oracle_model(p, g)
    tot = om.prepare(n_s, seed)
    rng = np.random.default_rng(seed)
    uids = np.sort(rng.choice(tot, size=min(400, tot), replace=False))
    lg, lo = gm.trace(n_s, seed, uids), om.run(uids=uids, log=True)["log"]
    r = compare_logs(lg, lo)
    assert r["n"] >= 0.99 * len(uids)
    assert len(r["flips"]) <= max(2, 0.01 * r["n"]), len(r["flips"])
    assert r["worst"]["X"] < 1e-8 and r["worst"]["K"] < 1e-8, r["worst"]
    # weights of recorded superphotons (an absorbed one may end at an FP32 underflow to 0 on one side)
    rec = compare_logs([x for x in lg if x["status"] == 1], [x for x in lo if x["status"] == 1])
    assert rec["n"] > 0 and rec["worst"]["w"] < 1e-3, rec["worst"]
