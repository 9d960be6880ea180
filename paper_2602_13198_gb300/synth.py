"""Seeded synthetic inputs (problem set-up only).

This module builds model dictionaries and fluid grids for the workloads of the
paper's tests (section 4) and their stand-ins.  It holds none of the transport
method's arithmetic: it only writes down the physical set-up (a static uniform
sphere with a vertical field, a Fishbone-Moncrief torus, lognormal turbulence) as
primitive variables on a grid.  Both the CUDA path and the CPU oracle consume
these dictionaries; neither is imported here.

Primitive layout: ``prim[8, n1*n2*n3]`` with fields (rho, u, B1, B2, B3, U1, U2, U3)
in code units, zone index ``(i*n2 + j)*n3 + k``.  ``U^i`` is the 4-velocity relative
to the normal observer, ``B^i`` the magnetic field 3-vector (HARM conventions),
both in the modified Kerr-Schild internal coordinates (x1 = ln r, x2, x3 = phi).
"""
from __future__ import annotations

import math

import numpy as np

# CGS constants used only to set up inputs (CODATA 2018 / IAU 2015 nominal GM_sun)
ME = 9.1093837015e-28
MP = 1.67262192369e-24
CL = 2.99792458e10
SIGMA_T = 6.6524587321e-25
GM_SUN = 1.3271244e26   # cm^3 s^-2
GAM = 13.0 / 9.0


def length_unit(m_bh_msun: float) -> float:
    """Gravitational radius GM/c^2 in cm."""
    return GM_SUN * m_bh_msun / (CL * CL)


def base_params(**over) -> dict:
    """Default model parameters (every field of the parameter structs)."""
    p = dict(
        a=0.0, mass=1.0, hslope=1.0,
        L_unit=length_unit(4e6), M_unit=1.0,
        R_high=1.0, R_low=1.0, gam=GAM,
        thetae_min=0.3, thetae_max=1000.0,
        nu_min=1e8, nu_max=1e16, w_min=1.0, n_s=1e5,
        eps_geo=0.04, verlet_tol=1e-3,
        r_record=1000.0, dh=0.05, bias_p0=1.0,
        lnu_lo=8.0, lnu_hi=24.0,
        roulette_w=1e-12, roulette_p=0.1,
        max_steps=20000,
        n_nu=200, verlet_maxit=16, bias_mode=0, n_sc_max=4,
        n_bins=200, n_incl=1, k2_mode=0, scatter=0,
    )
    p.update(over)
    return p


def _grid(n1, n2, n3, x1_0, x1_1):
    return dict(n1=n1, n2=n2, n3=n3,
                x1_0=x1_0, dx1=(x1_1 - x1_0) / n1,
                x2_0=0.0, dx2=1.0 / n2,
                x3_0=0.0, dx3=2.0 * math.pi / n3)


def _zone_centres(g):
    i = np.arange(g["n1"])
    j = np.arange(g["n2"])
    k = np.arange(g["n3"])
    x1 = g["x1_0"] + (i + 0.5) * g["dx1"]
    x2 = g["x2_0"] + (j + 0.5) * g["dx2"]
    x3 = g["x3_0"] + (k + 0.5) * g["dx3"]
    X1, X2, X3 = np.meshgrid(x1, x2, x3, indexing="ij")
    return X1.ravel(), X2.ravel(), X3.ravel()


def sphere(metric: str = "ks", *, R: float = 10.0, n1: int = 1024, n2: int = 128,
           ne: float = 1e13, thetae: float = 10.0, B_gauss: float = 10.0,
           m_bh_msun: float = 4e6, L_unit: float | None = None, r_in: float | None = None,
           dh: float = 0.05, **over):
    """Uniform static sphere with a vertical magnetic field (section 4.1 set-up).

    ``metric='ks'``: Schwarzschild (a = 0) in Kerr-Schild form with the hole at the
    centre; the grid spans ln r in [ln(r_h (1 + dh)), ln R] so the sphere edge is a
    grid edge.  The fluid is at rest (static observers) and the field has fluid-frame
    strength ``B_gauss`` along the static frame's vertical direction.
    ``metric='flat'``: Minkowski space (the paper's analytic test), grid ln r in
    [ln r_in, ln R].
    Density and temperature: rho = 1 with M_unit chosen so that n_e = ``ne``;
    R_high = R_low = 1 and u/rho chosen so the temperature model gives ``thetae``.
    """
    flat = metric == "flat"
    if L_unit is None:
        L_unit = 1.0 if flat else length_unit(m_bh_msun)
    if flat:
        r0 = r_in if r_in is not None else 1e-3 * R
    else:
        r0 = 2.0 * (1.0 + dh)
    g = _grid(n1, n2, 1, math.log(r0), math.log(R))
    X1, X2, _ = _zone_centres(g)
    r = np.exp(X1)
    th = math.pi * X2
    rho_unit = ne * (MP + ME)
    M_unit = rho_unit * L_unit ** 3
    B_unit = CL * math.sqrt(4.0 * math.pi * rho_unit)
    B0 = B_gauss / B_unit
    nz = r.size
    prim = np.zeros((8, nz))
    prim[0] = 1.0
    # Theta_e = (m_p/m_e) (gam - 1) (u/rho) / (1 + T_i/T_e) with T_i/T_e = 1
    prim[1] = 2.0 * thetae * ME / (MP * (GAM - 1.0))
    if flat:
        # at rest: U^i = 0; B^i = b^i; b = B0 z-hat = B0 (cos th e_r - sin th e_th)
        prim[2] = B0 * np.cos(th) / r                 # B^{x1} = B^r / r
        prim[3] = -B0 * np.sin(th) / r / math.pi      # B^{x2} = B^th / (dth/dx2)
    else:
        f = 1.0 - 2.0 / r
        # static observer in Schwarzschild-KS: u^t = f^-1/2, u^i = 0.
        # normal-observer velocity U^r = gamma alpha g^{tr}, alpha = (1 + 2/r)^-1/2,
        # gamma = alpha u^t, g^{tr} = 2/r; in x1 = ln r: U^{x1} = U^r / r.
        alpha = 1.0 / np.sqrt(1.0 + 2.0 / r)
        gamma = alpha / np.sqrt(f)
        prim[5] = gamma * alpha * (2.0 / r) / r
        # fluid-frame field B0 (cos th e_r^ - sin th e_th^); B^i = b^i u^t for u^i = 0:
        # b^r = B0 cos th f^1/2, b^th = -B0 sin th / r  ->  B^r = B0 cos th, B^th = -B0 sin th / (r f^1/2)
        prim[2] = B0 * np.cos(th) / r
        prim[3] = -B0 * np.sin(th) / (r * np.sqrt(f)) / math.pi
    params = base_params(
        mass=0.0 if flat else 1.0, a=0.0, hslope=1.0, L_unit=L_unit, M_unit=M_unit,
        R_high=1.0, R_low=1.0, dh=dh)
    params.update(over)
    g["prim"] = prim
    return params, g


def scattering_sphere(tau_t: float, *, R: float = 10.0, thetae: float = 4.0, **over):
    """Scattering sphere (section 4.2 set-up, Schwarzschild): n_e from the Thomson
    depth tau_T = n_e sigma_T R; constant bias b = max(1, 0.01 / (3/4 tau_T)), so that
    about one primary in a hundred scatters (the mean escape chord of a uniform
    isotropic emitter is 3R/4)."""
    L = length_unit(4e6)
    ne = tau_t / (SIGMA_T * R * L)
    bias = 0.01 / (0.75 * tau_t)
    kw = dict(scatter=1, bias_mode=0, bias_p0=bias, n_sc_max=4)
    kw.update(over)
    return sphere("ks", R=R, ne=ne, thetae=thetae, **kw)
