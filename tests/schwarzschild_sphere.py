"""Deterministic reference for the optically thin bins of the uniform static sphere in the
Schwarzschild metric (the bench's config-1 sphere): for a static emitter at radius r (units of M)
the energy at infinity is E f(r), f = (1 - 2/r)^1/2, and with the KS volume element
sqrt(-g) = r^2 sin(theta) the luminosity per unit frequency at infinity is
    L_nu(nu_inf) = L^3 int r^2 dr int sin(theta) dtheta int dphi int dOmega_n j(nu_inf / f, cos theta_B) 1_esc,
with n the emission direction in the static frame, psi its angle to e_r, theta_B its angle to the
vertical field z = cos(theta) e_r - sin(theta) e_theta.  Capture rule for photons (impact parameter
b = r sin(psi) / f against 3 sqrt 3): the escaping directions are psi in [0, psi_max(r)] with
psi_max = pi - arcsin(s) for r >= 3 and arcsin(s) for r < 3, s = 3 sqrt(3) f / r."""
import math

import numpy as np
from scipy import special

EE, ME, CL = 4.803204712570263e-10, 9.1093837015e-28, 2.99792458e10   # CODATA 2018 (exact e in statC)


def jnu(nu, c, ne, thetae, B, nu_lo, nu_hi):
    """Thermal synchrotron emissivity (the paper's fit, eq. emissivity) with exact K2; zero outside
    the emission band [nu_lo, nu_hi] and along the field."""
    s = np.sqrt(np.clip(1.0 - c * c, 0.0, 1.0))
    nus = (2.0 / 9.0) * (EE * B / (2.0 * math.pi * ME * CL)) * thetae ** 2 * s
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        X = nu / nus
        t = np.sqrt(X) + 2.0 ** (11.0 / 12.0) * X ** (1.0 / 6.0)
        j = math.sqrt(2.0) * math.pi * EE ** 2 * ne * nus / (3.0 * CL * special.kv(2, 1.0 / thetae)) * t * t * np.exp(-np.cbrt(X))
    j = np.where((s > 0) & (nu >= nu_lo) & (nu <= nu_hi), j, 0.0)
    return np.nan_to_num(j)


def _gl(n, a, b):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def angular_measure(r, gravity=True, n_th=64, n_psi=64, n_chi=32, n_c=4096):
    """Weights H[m] on the grid c_m of cos(theta_B) such that int sin(theta) dtheta dOmega_n 1_esc g(cos theta_B)
    ~ sum_m H[m] g(c_m) for smooth g (linear deposit); the phi integral (2 pi) is left out."""
    f = math.sqrt(1.0 - 2.0 / r) if gravity else 1.0
    if gravity:
        s = min(1.0, 3.0 * math.sqrt(3.0) * f / r)
        psi_max = math.pi - math.asin(s) if r >= 3.0 else math.asin(s)
    else:
        psi_max = math.pi
    th, wth = _gl(n_th, 0.0, math.pi)
    ps, wps = _gl(n_psi, 0.0, psi_max)
    ch, wch = _gl(n_chi, 0.0, math.pi)
    T, P, Ch = np.meshgrid(th, ps, ch, indexing="ij")
    W = (np.sin(T) * wth[:, None, None]) * (np.sin(P) * wps[None, :, None]) * (2.0 * wch[None, None, :])
    c = np.cos(P) * np.cos(T) - np.sin(P) * np.cos(Ch) * np.sin(T)
    grid = np.linspace(-1.0, 1.0, n_c)
    pos = (np.clip(c.ravel(), -1.0, 1.0) + 1.0) / 2.0 * (n_c - 1)
    i0 = np.minimum(np.floor(pos).astype(int), n_c - 2)
    fr = pos - i0
    H = np.zeros(n_c)
    np.add.at(H, i0, W.ravel() * (1.0 - fr))
    np.add.at(H, i0 + 1, W.ravel() * fr)
    return grid, H, f


def nuLnu_bins(p, r_in, R, ne, thetae, B, bins, gravity=True, n_r=64, n_nu=4):
    """Bin averages over ln(nu_inf) of nu L_nu [erg/s] for the listed bin indices."""
    dlog = (p["lnu_hi"] - p["lnu_lo"]) / p["n_bins"]
    rs, wr = _gl(n_r, r_in, R)
    meas = [angular_measure(r, gravity) for r in rs]
    xg, wg = np.polynomial.legendre.leggauss(n_nu)
    out = []
    for b in bins:
        lo = p["lnu_lo"] + b * dlog
        lg = lo + 0.5 * dlog * (xg + 1.0)
        acc = 0.0
        for (grid, H, f), r, w in zip(meas, rs, wr):
            nu_inf = 10.0 ** lg
            J = jnu(nu_inf[:, None] / f, grid[None, :], ne, thetae, B, p["nu_min"], p["nu_max"])
            L = 2.0 * math.pi * r * r * w * (J @ H) * p["L_unit"] ** 3
            acc += np.sum(0.5 * wg * nu_inf * L)
        out.append(acc)
    return np.array(out)
