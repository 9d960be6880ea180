"""Pins of the oracle's fluid state, plasma-frame tetrads and fluid interpolation (sections 2.1,
2.2, 2.5 and 2.7; the readings on coordinates, temperature model and interpolation).

Each check is computed here without the oracle's formulas, at random points of spinning tori
(a = 0.9375 and the retrograde a = -0.94) with every primitive component non-zero:
- u^mu: normalised (u.u = -1), and its part orthogonal to the normal observer n (n_mu = (-alpha, 0,
  0, 0)) is the primitive velocity U^i, with gamma = -n.u = sqrt(1 + U.U);
- b^mu: the solution of the linear system b.u = 0, b^i u^t - b^t u^i = B^i (the ideal-MHD dual
  field *F^{i t} = B^i), solved by numpy; b^2 also against (B^2 + (B.u)^2) / (u^t)^2; in the frame of
  the normal observer (U = 0) b^2 = alpha^2 g_ij B^i B^j;
- n_e and |B| from the unit definitions, Theta_e at the three points of the temperature model that
  fix it: beta -> infinity (no field: R_high), beta = 1 (the mean of R_high and R_low) and beta -> 0
  (strong field: R_low), where beta = (gamma_hat - 1) u / (b^2 / 2);
- tetrads: e_a . e_b = eta_ab, e_0 = u, e_3 = b / |b| (emission), and the scattering tetrad's
  Gram-Schmidt structure (e_k in the span of u, d_1 .. d_k with a positive d_k component);
- fluid_at: a primitive field linear in (x1, x2, x3) is reproduced exactly between zone centres,
  held at the edge value beyond the outer centres in x1 and x2, blended across the periodic seam in
  x3, and switched off outside the radial extent of the grid.
A wrong lapse, a sign in b^mu, beta from b^2 instead of b^2 / 2, R_high and R_low swapped, or an
interpolation weight off by a zone fails one of these."""
import math

import numpy as np
import pytest

from paper_2602_13198_gb300 import synth

MP_ME = 1836.15267343        # proton-electron mass ratio (CODATA 2018)
ME, MP, CL = 9.1093837015e-28, 1.67262192369e-24, 2.99792458e10
ETA = np.diag([-1.0, 1.0, 1.0, 1.0])


def random_states(a, n=100, seed=3):
    """Points (X, primitives) drawn from zones of a torus grid with every component perturbed."""
    p, g = synth.torus(a=a, n1=64, n2=32, seed=7)
    rng = np.random.default_rng(seed)
    prim = np.asarray(g["prim"], dtype=np.float64)
    nz = prim.shape[1]
    out = []
    x1_lo, x1_hi = g["x1_0"], g["x1_0"] + g["n1"] * g["dx1"]
    for _ in range(n):
        z = int(rng.integers(nz))
        pr = prim[:, z].copy()
        X = np.array([0.0, rng.uniform(x1_lo + 0.3, x1_hi), rng.uniform(0.03, 0.97), rng.uniform(0, 2 * math.pi)])
        bscale = max(float(np.max(np.abs(pr[2:5]))), 1e-3)
        pr[2:5] += rng.normal(0.0, bscale, 3) * np.array([1.0, 1.0, 0.5])
        pr[5:8] += rng.normal(0.0, 0.2, 3) * np.array([0.3, 0.5, 0.05])
        pr[0] = abs(pr[0]) + 1e-3
        pr[1] = abs(pr[1]) + 1e-5
        out.append((X, pr))
    return p, out


def normal_observer(g):
    gi = np.linalg.inv(g)
    alpha = 1.0 / math.sqrt(-gi[0, 0])
    n_up = -alpha * gi[:, 0]
    return alpha, n_up


def b_from_linear_system(ucon, ucov, B):
    A = np.zeros((4, 4))
    rhs = np.zeros(4)
    A[0, :] = ucov
    for i in (1, 2, 3):
        A[i, 0] = -ucon[i]
        A[i, i] = ucon[0]
        rhs[i] = B[i - 1]
    return np.linalg.solve(A, rhs)


@pytest.mark.parametrize("a", [0.9375, -0.94])
def test_four_velocity_and_field_at_random_torus_points(oracle_mod, a):
    cfg, pts = random_states(a)
    rho_unit = cfg["M_unit"] / cfg["L_unit"] ** 3
    B_unit = CL * math.sqrt(4 * math.pi * rho_unit)
    for X, pr in pts:
        g = oracle_mod.gcov(cfg, X)
        f = oracle_mod.fluid_from_prims(cfg, X, pr)
        u, ul = f["ucon"], f["ucov"]
        assert np.allclose(ul, g @ u, rtol=1e-13, atol=1e-13 * np.max(np.abs(ul)))
        assert u @ g @ u == pytest.approx(-1.0, abs=1e-12)
        alpha, n_up = normal_observer(g)
        U = pr[5:8]
        gamma = math.sqrt(1.0 + U @ g[1:, 1:] @ U)
        assert alpha * u[0] == pytest.approx(gamma, rel=1e-12)          # -n.u with n_mu = (-alpha, 0, 0, 0)
        proj = u - gamma * n_up
        assert abs(proj[0]) <= 1e-12 * max(1.0, np.max(np.abs(u)))
        assert np.allclose(proj[1:], U, rtol=1e-11, atol=1e-12 * max(1.0, np.max(np.abs(u))))
        # magnetic 4-vector
        bref = b_from_linear_system(u, ul, pr[2:5])
        scale = np.max(np.abs(bref)) + 1e-300
        assert np.allclose(f["bcon"], bref, rtol=1e-10, atol=1e-11 * scale)
        assert np.allclose(f["bcov"], g @ f["bcon"], rtol=1e-12, atol=1e-12 * np.max(np.abs(f["bcov"])))
        assert abs(f["bcon"] @ ul) <= 1e-11 * scale * np.max(np.abs(ul))
        Bv = np.concatenate([[0.0], pr[2:5]])
        bsq = ((Bv @ g @ Bv) + (Bv @ ul) ** 2) / u[0] ** 2
        assert f["bsq"] == pytest.approx(bsq, rel=1e-10)
        assert f["B"] == pytest.approx(math.sqrt(bsq) * B_unit, rel=1e-10)
        assert f["ne"] == pytest.approx(pr[0] * rho_unit / (MP + ME), rel=1e-13)


@pytest.mark.parametrize("a", [0.9375, -0.94])
def test_field_in_the_normal_observer_frame(oracle_mod, a):
    cfg, pts = random_states(a, n=30, seed=5)
    for X, pr in pts:
        pr = pr.copy()
        pr[5:8] = 0.0
        g = oracle_mod.gcov(cfg, X)
        f = oracle_mod.fluid_from_prims(cfg, X, pr)
        alpha, n_up = normal_observer(g)
        assert np.allclose(f["ucon"], n_up, rtol=1e-12, atol=1e-14)
        B = pr[2:5]
        assert f["bsq"] == pytest.approx(alpha ** 2 * (B @ g[1:, 1:] @ B), rel=1e-11)


@pytest.mark.parametrize("a", [0.9375, -0.94])
def test_electron_temperature_limits(oracle_mod, a):
    cfg, pts = random_states(a, n=30, seed=11)
    cfg = dict(cfg, R_high=20.0, R_low=1.0, thetae_max=1e30)
    gam = cfg["gam"]
    for X, pr in pts:
        pr = pr.copy()
        base = MP_ME * (gam - 1.0) * pr[1] / pr[0]
        # no field: beta infinite, T_i/T_e = R_high
        p0 = pr.copy()
        p0[2:5] = 0.0
        assert oracle_mod.fluid_from_prims(cfg, X, p0)["thetae"] == pytest.approx(base / (1 + 20.0), rel=1e-10)
        # beta = 1 exactly: b^2 / 2 = (gamma_hat - 1) u, T_i/T_e = (R_high + R_low) / 2
        g = oracle_mod.gcov(cfg, X)
        f = oracle_mod.fluid_from_prims(cfg, X, pr)
        Bv = np.concatenate([[0.0], pr[2:5]])
        bsq1 = ((Bv @ g @ Bv) + (Bv @ f["ucov"]) ** 2) / f["ucon"][0] ** 2
        p1 = pr.copy()
        p1[2:5] *= math.sqrt(2.0 * (gam - 1.0) * pr[1] / bsq1)
        assert oracle_mod.fluid_from_prims(cfg, X, p1)["thetae"] == pytest.approx(base / (1 + 10.5), rel=1e-9)
        # strong field: beta -> 0, T_i/T_e -> R_low
        p2 = pr.copy()
        p2[2:5] *= 1e6 * math.sqrt(2.0 * (gam - 1.0) * pr[1] / bsq1)
        assert oracle_mod.fluid_from_prims(cfg, X, p2)["thetae"] == pytest.approx(base / (1 + 1.0), rel=1e-9)


def test_thetae_ceiling_and_empty_zone(oracle_mod):
    cfg, pts = random_states(0.9375, n=5, seed=2)
    X, pr = pts[0]
    pr = pr.copy()
    pr[1] = 10.0 * pr[0]          # Theta_e of several hundred without the ceiling
    cfg = dict(cfg, thetae_max=0.5)
    assert oracle_mod.fluid_from_prims(cfg, X, pr)["thetae"] == 0.5
    pr[0] = 0.0
    f = oracle_mod.fluid_from_prims(cfg, X, pr)
    assert f["ne"] == 0.0 and f["thetae"] == 0.0


@pytest.mark.parametrize("a", [0.9375, -0.94])
def test_tetrads_are_orthonormal_plasma_frames(oracle_mod, a):
    cfg, pts = random_states(a, n=100, seed=17)
    for X, pr in pts:
        g = oracle_mod.gcov(cfg, X)
        f = oracle_mod.fluid_from_prims(cfg, X, pr)
        for kind in ("emission", "scatter"):
            e = oracle_mod.tetrad(cfg, X, pr, kind)
            gram = e @ g @ e.T
            assert np.allclose(gram, ETA, atol=1e-11), (kind, gram)
            assert np.allclose(e[0], f["ucon"], rtol=1e-14, atol=0)
        e = oracle_mod.tetrad(cfg, X, pr, "emission")
        bn = f["bcon"] / math.sqrt(f["bsq"])
        assert np.allclose(e[3], bn, rtol=1e-12, atol=1e-12 * np.max(np.abs(bn)))
        # scattering tetrad: e_k in span(u, d_1 .. d_k) with g(e_k, d_k) > 0
        e = oracle_mod.tetrad(cfg, X, pr, "scatter")
        for k in (1, 2, 3):
            basis = [f["ucon"]] + [np.eye(4)[j] for j in range(1, k + 1)]
            M = np.array(basis).T
            coef, *_ = np.linalg.lstsq(M, e[k], rcond=None)
            assert np.allclose(M @ coef, e[k], atol=1e-11 * np.max(np.abs(e[k])))
            assert (e[k] @ g)[k] > 0.0


def linear_grid(a):
    """A small MKS grid whose primitives are linear in (x1, x2, x3)."""
    n1, n2, n3 = 8, 6, 5
    rh = 1.0 + math.sqrt(1.0 - a * a)
    g = dict(n1=n1, n2=n2, n3=n3, x1_0=math.log(rh) + 0.2, dx1=0.25, x2_0=0.1, dx2=0.8 / n2,
             x3_0=0.3, dx3=2 * math.pi / n3)
    C = np.array([[1.0, 0.05, 0.3, 0.02], [0.5, 0.04, -0.1, 0.01], [0.02, 0.003, -0.01, 0.002],
                  [-0.01, 0.002, 0.015, -0.001], [0.005, -0.001, 0.002, 0.0005], [0.05, 0.01, -0.02, 0.003],
                  [0.01, -0.002, 0.01, 0.001], [0.08, -0.01, 0.02, 0.002]])
    x1 = g["x1_0"] + (np.arange(n1) + 0.5) * g["dx1"]
    x2 = g["x2_0"] + (np.arange(n2) + 0.5) * g["dx2"]
    x3 = g["x3_0"] + (np.arange(n3) + 0.5) * g["dx3"]
    X1, X2, X3 = np.meshgrid(x1, x2, x3, indexing="ij")
    prim = np.stack([C[f, 0] + C[f, 1] * X1 + C[f, 2] * X2 + C[f, 3] * X3 for f in range(8)]).reshape(8, -1)
    g["prim"] = prim
    cfg = synth.base_params(a=a, hslope=0.3, M_unit=1e18, R_high=20.0, L_unit=synth.length_unit(4.14e6))
    return cfg, g, C, (x1, x2, x3)


def _prims(C, x1, x2, x3):
    return C[:, 0] + C[:, 1] * x1 + C[:, 2] * x2 + C[:, 3] * x3


def _same_state(fa, fb):
    for k in ("ne", "thetae", "B"):
        assert fa[k] == pytest.approx(fb[k], rel=1e-11, abs=1e-300), k
    for k in ("ucon", "bcon"):
        s = np.max(np.abs(fb[k])) + 1e-300
        assert np.allclose(fa[k], fb[k], rtol=1e-11, atol=1e-12 * s), k


@pytest.mark.parametrize("a", [0.5, -0.94])
def test_fluid_at_reproduces_a_linear_field(oracle_mod, a):
    cfg, g, C, (x1c, x2c, x3c) = linear_grid(a)
    om = oracle_mod.Model(cfg, g)
    rng = np.random.default_rng(23)
    for _ in range(60):   # between zone centres: exact
        X = np.array([0.0, rng.uniform(x1c[0], x1c[-1]), rng.uniform(x2c[0], x2c[-1]), rng.uniform(x3c[0], x3c[-1])])
        fa = om.fluid(X)
        assert fa["plasma"]
        _same_state(fa, oracle_mod.fluid_from_prims(cfg, X, _prims(C, *X[1:])))
    lo1, hi1 = g["x1_0"], g["x1_0"] + g["n1"] * g["dx1"]
    for _ in range(20):   # beyond the outer centres in x1 and x2: held at the edge centre's value
        x1 = rng.choice([rng.uniform(lo1, x1c[0]), rng.uniform(x1c[-1], hi1)])
        x2 = rng.choice([rng.uniform(0.01, x2c[0]), rng.uniform(x2c[-1], 0.99)])
        x3 = rng.uniform(x3c[0], x3c[-1])
        X = np.array([0.0, x1, x2, x3])
        xe1 = min(max(x1, x1c[0]), x1c[-1])
        xe2 = min(max(x2, x2c[0]), x2c[-1])
        _same_state(om.fluid(X), oracle_mod.fluid_from_prims(cfg, X, _prims(C, xe1, xe2, x3)))
    for _ in range(20):   # across the periodic seam in x3: blend of the last and the first zone
        x1, x2 = rng.uniform(x1c[0], x1c[-1]), rng.uniform(x2c[0], x2c[-1])
        x3 = rng.uniform(x3c[-1], x3c[0] + 2 * math.pi)
        d = (x3 - x3c[-1]) / g["dx3"]
        pr = (1 - d) * _prims(C, x1, x2, x3c[-1]) + d * _prims(C, x1, x2, x3c[0])
        X = np.array([0.0, x1, x2, x3 if x3 < g["x3_0"] + 2 * math.pi else x3 - 2 * math.pi])
        _same_state(om.fluid(X), oracle_mod.fluid_from_prims(cfg, X, pr))
    for x1 in (lo1 - 0.05, hi1 + 0.05):   # outside the radial extent: no plasma
        fa = om.fluid(np.array([0.0, x1, 0.5, 1.0]))
        assert not fa["plasma"] and fa["ne"] == 0.0
