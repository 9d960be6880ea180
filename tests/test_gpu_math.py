"""The library's own special-function implementations against CUDA's on the device: the Taylor
sine/cosine of the small theta-map angle (metric evaluation), the Newton x^(1/6) of the
synchrotron function, the double-float e^x and sin/cos(pi x) of the mixed-precision geodesic, and the
table-driven FP64 e^x, ln x and sin/cos(pi x) of the FP64 transport (after Tang 1989, 1990)."""
import numpy as np
import pytest

from helpers import requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _mc():
    from paper_2602_13198_gb300 import build, mc
    build.build()
    return mc


def test_small_angle_sine_and_cosine_match_cuda():
    mc = _mc()
    x = np.concatenate([np.linspace(-0.5, 0.5, 200001), np.array([0.0, 1e-300, -1e-12, 0.35, -0.35])])
    s, s_ref = mc.selftest_math(0, x)
    c, c_ref = mc.selftest_math(1, x)
    # a few units in the last place of the result
    assert np.all(np.abs(s - s_ref) <= 4 * np.spacing(np.abs(s_ref)) + 1e-300)
    assert np.all(np.abs(c - c_ref) <= 4 * np.spacing(np.abs(c_ref)))
    # the exact small-argument behaviour: sin x = x, cos x = 1
    assert s[-4] == 1e-300 and c[-4] == 1.0


def test_sixth_root_matches_cuda():
    mc = _mc()
    rng = np.random.default_rng(4)
    x = np.concatenate([10.0 ** rng.uniform(-29.9, 29.9, 200000),
                        np.array([1.0, 64.0, 1e-30, 1e30, 1e-40, 1e40, 3.0e-31, 7.0e35])])
    y, ref = mc.selftest_math(2, x)
    rel = np.abs(y / ref - 1.0)
    # X z^5 takes four roundings after the Newton steps, cbrt(sqrt(x)) two: within 10 ulp
    assert rel.max() < 10 * 2.2e-16, rel.max()
    assert abs(y[-8] - 1.0) <= 2.3e-16 and abs(y[-7] - 2.0) <= 4.5e-16   # x = 1 and x = 64


def test_double_float_exp_matches_cuda():
    mc = _mc()
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(-20.0, 20.0, 200000), np.linspace(-0.02, 0.02, 4001),
                        np.array([0.0, 1.0, np.log(2.0), 0.6931471805599453 / 64, 10.0, -10.0])])
    y, ref = mc.selftest_math(3, x)
    rel = np.abs(y / ref - 1.0)
    # 48-bit arithmetic: the reduction x - k ln2/32 carries |x| 2^-48 of absolute error
    bound = 4.0 * 2.0 ** -48 * np.maximum(1.0, np.abs(x))
    assert np.all(rel <= bound), (rel / bound).max()
    assert y[-6] == 1.0


@pytest.mark.parametrize("which", [4, 5])
def test_double_float_sincospi_matches_cuda(which):
    mc = _mc()
    rng = np.random.default_rng(6 + which)
    x = np.concatenate([rng.uniform(-2.0, 3.0, 200000), np.arange(-64, 97) / 32.0,
                        np.array([1e-9, 0.5 - 1e-12, 1.0 - 1e-15])])
    y, ref = mc.selftest_math(which, x)
    assert np.abs(y - ref).max() <= 4.0 * 2.0 ** -48
    # exact at multiples of 1/2
    k = np.arange(-64, 97) / 32.0
    half = (np.abs(k * 2 - np.round(k * 2)) == 0)
    yk = y[200000:200000 + len(k)]
    assert np.all(np.isin(np.abs(yk[half]), [0.0, 1.0]))


def test_table_driven_exp_matches_cuda():
    mc = _mc()
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.uniform(-707.9, 707.9, 200000), rng.uniform(-1.0, 1.0, 100000),
                        np.linspace(-0.011, 0.011, 4001),
                        np.array([0.0, 1.0, -1.0, np.log(2.0), 707.9, -707.9, 708.0, -708.0, 709.5, -745.0, -800.0])])
    y, ref = mc.selftest_math(6, x)
    fin = ref > 0
    rel = np.abs(y[fin] / ref[fin] - 1.0)
    # within 3 ulp of CUDA's exp; outside (-708, 708) the function is CUDA's own
    assert rel.max() <= 3 * 2.2e-16, rel.max()
    assert y[-11] == 1.0 and np.array_equal(y[-5:], ref[-5:])


def test_table_driven_expm1_matches_cuda():
    mc = _mc()
    rng = np.random.default_rng(14)
    x = np.concatenate([rng.uniform(-0.25, 0.25, 200000), rng.uniform(-40.0, 40.0, 200000),
                        10.0 ** rng.uniform(-300, -1, 50000) * rng.choice([-1.0, 1.0], 50000),
                        np.linspace(0.2499, 0.2501, 2001), np.linspace(-0.2501, -0.2499, 2001),
                        np.array([0.0, -0.0, 0.25, -0.25, 1e-300, 700.0, -700.0, -800.0, 800.0])])
    y, ref = mc.selftest_math(10, x)
    fin = np.isfinite(ref) & (ref != 0.0)
    rel = np.abs(y[fin] / ref[fin] - 1.0)
    # the series below |x| = 1/4 within 3 ulp of CUDA's expm1; above it e^x - 1 from exp_t (within
    # 3 ulp of CUDA's exp) loses at most ~2.2 bits to the subtraction: 3 ulp x 4.5 < 3e-15
    small = np.abs(x[fin]) < 0.25
    assert rel[small].max() <= 3 * 2.2e-16, rel[small].max()
    assert rel[~small].max() <= 3e-15, rel[~small].max()
    assert y[-9] == 0.0 and y[-8] == 0.0 and y[-5] == 1e-300
    assert y[-2] == -1.0 and np.isinf(y[-1]) and y[-1] > 0


def test_table_driven_log_matches_cuda():
    mc = _mc()
    rng = np.random.default_rng(12)
    x = np.concatenate([10.0 ** rng.uniform(-300, 300, 200000), rng.uniform(0.5, 2.0, 100000),
                        1.0 + np.linspace(-1e-6, 1e-6, 2001),
                        np.array([1.0, 2.0, 0.5, 1e-310, 0.0, 1e308])])
    y, ref = mc.selftest_math(7, x)
    big = np.isfinite(ref) & (np.abs(ref) >= 1e-2)
    # ~1 ulp away from x = 1: within 4 ulp of CUDA's log; near x = 1 within 3e-16 absolute
    assert (np.abs(y[big] - ref[big]) / np.abs(ref[big])).max() <= 4 * 2.2e-16
    assert np.abs(y[~big & np.isfinite(ref)] - ref[~big & np.isfinite(ref)]).max() <= 3e-16
    assert y[-6] == 0.0 and y[-2] == ref[-2] and y[-3] == ref[-3]   # ln 1 = 0; subnormal and 0 take CUDA's log


@pytest.mark.parametrize("which", [8, 9])
def test_table_driven_sincospi_matches_cuda(which):
    mc = _mc()
    rng = np.random.default_rng(13 + which)
    x = np.concatenate([rng.uniform(-2.0, 3.0, 200000), rng.uniform(0.0, 1.0, 100000), np.arange(-64, 97) / 32.0,
                        np.array([1e-9, 0.5 - 1e-12, 1.0 - 1e-15, 1e-300])])
    y, ref = mc.selftest_math(which, x)
    assert np.abs(y - ref).max() <= 3 * 2.2e-16
    k = np.arange(-64, 97) / 32.0
    half = (np.abs(k * 2 - np.round(k * 2)) == 0)
    yk = y[300000:300000 + len(k)]
    assert np.all(np.isin(np.abs(yk[half]), [0.0, 1.0]))
    if which == 8:
        assert y[-1] == np.pi * 1e-300 or abs(y[-1] / (np.pi * 1e-300) - 1) < 1e-15

