"""Oracle pins: counter-based random numbers and quadrature rules."""
import numpy as np
from conftest import golden


def test_philox_known_answers(oracle_mod):
    # Salmon et al. 2011 known-answer vectors (tests/golden/philox4x32_10_kat.txt)
    for row in golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        assert oracle_mod.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniforms_open_interval_and_streams(oracle_mod):
    u = oracle_mod.uniforms(1, 7, 200000)
    assert np.all(u > 0.0) and np.all(u < 1.0)
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / u.size)
    # uniform histogram (chi^2 with 50 bins)
    h, _ = np.histogram(u, bins=50, range=(0, 1))
    e = u.size / 50
    chi2 = ((h - e) ** 2 / e).sum()
    assert chi2 < 49 + 5 * np.sqrt(2 * 49)
    # different streams / seeds give different sequences; draws are a pure function of (seed, id, n)
    assert not np.allclose(u[:10], oracle_mod.uniforms(1, 8, 10))
    assert not np.allclose(u[:10], oracle_mod.uniforms(2, 7, 10))
    assert np.array_equal(u[5:15], oracle_mod.uniforms(1, 7, 10, start=5))


def test_uniform_bits_from_philox_words(oracle_mod):
    # draw n uses Philox block n//2 (counter = (n//2, 0, id_lo, id_hi), key = (seed_lo, seed_hi)),
    # words (0,1) for even n and (2,3) for odd n; u = ((a << 21 | b >> 11) + 1/2) 2^-53
    seed, sid = 0x123456789ABCDEF, 0xFEDCBA9876543210
    u = oracle_mod.uniforms(seed, sid, 4)
    for n in range(4):
        o = oracle_mod.philox([n >> 1, 0, sid & 0xFFFFFFFF, sid >> 32], [seed & 0xFFFFFFFF, seed >> 32])
        a, b = (o[2], o[3]) if n & 1 else (o[0], o[1])
        m = (a << 21) | (b >> 11)
        assert u[n] == (m + 0.5) * 2.0 ** -53


def test_child_stream_is_splitmix64(oracle_mod):
    # splitmix64 (Steele, Lea & Flood 2014) written out with Python integers
    def splitmix64(state):
        z = state & (2**64 - 1)
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & (2**64 - 1)
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & (2**64 - 1)
        return z ^ (z >> 31)
    for parent, ev in [(0, 0), (12345, 3), (2**63 + 5, 7)]:
        assert oracle_mod.child_stream(parent, ev) == splitmix64(parent + 0x9E3779B97F4A7C15 * (ev + 1))


def test_gauss_legendre_moments(oracle_mod):
    for n in (8, 32, 64):
        x, w = oracle_mod.gauss_legendre(n, 0.0, 2.0)
        for k in range(2 * n):
            exact = 2.0 ** (k + 1) / (k + 1)
            assert abs((w * x**k).sum() - exact) <= 1e-12 * exact
        ref_x, _ = np.polynomial.legendre.leggauss(n)
        assert np.allclose(np.sort(x), np.sort(ref_x + 1.0), rtol=0, atol=1e-13)
