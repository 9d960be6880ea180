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
        roulette_w=1e-12, roulette_p=0.1, bias_max=1e300, bias_target=0.0, kappa=0.0, brems=0,
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


def inside_fraction(g, R, sub):
    """Fraction of each zone inside r < R (section 4.1 partial cells): the zone is split into
    sub x sub sub-cells in (x1, x2) and the sub-cell centres with r = exp(x1) < R are counted.
    sub = 0: 1 for zones whose centre lies inside, else 0 (an abrupt edge)."""
    X1, X2, _ = _zone_centres(g)
    if sub == 0:
        return (np.exp(X1) < R).astype(float)
    off = (np.arange(sub) + 0.5) / sub - 0.5
    x1s = X1[:, None] + off[None, :] * g["dx1"]
    # a sphere's edge depends on r only, so the x2 sub-cells repeat the same count sub times
    inside = (np.exp(x1s) < R).sum(axis=1) * sub
    return inside / float(sub * sub)


def sphere(metric: str = "ks", *, R: float = 10.0, n1: int = 1024, n2: int = 128,
           ne: float = 1e13, thetae: float = 10.0, B_gauss: float = 10.0,
           m_bh_msun: float = 4e6, L_unit: float | None = None, r_in: float | None = None,
           dh: float = 0.05, r_out: float | None = None, partial: int = 0, **over):
    """Uniform static sphere with a vertical magnetic field (section 4.1 set-up).

    ``metric='ks'``: Schwarzschild (a = 0) in Kerr-Schild form with the hole at the
    centre; the grid spans ln r in [ln(r_h (1 + dh)), ln R] so the sphere edge is a
    grid edge.  The fluid is at rest (static observers) and the field has fluid-frame
    strength ``B_gauss`` along the static frame's vertical direction.
    ``metric='flat'``: Minkowski space (the paper's analytic test), grid ln r in
    [ln r_in, ln R].
    ``r_out`` > R extends the grid beyond the sphere (the paper's 10^4 cm), with no gas outside
    R: rho and u of each zone are scaled by its inside fraction (``inside_fraction`` with
    ``partial`` sub-cells per side; 0 = the zone centre decides), which keeps Theta_e.
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
    r1 = R if r_out is None else r_out
    g = _grid(n1, n2, 1, math.log(r0), math.log(r1))
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
    if r1 > R:
        frac = inside_fraction(g, R, partial)
        prim[0] *= frac
        prim[1] *= frac
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


# ----------------------------------------------------------------------------- tori (section 4.3 stand-ins)
def _ks_mks_metric(r, th, dth, a):
    """Covariant Kerr-Schild metric (M = 1) in MKS internal coordinates, as [..., 4, 4] (set-up use)."""
    s2, c2 = np.sin(th) ** 2, np.cos(th) ** 2
    sig = r * r + a * a * c2
    f = 2.0 * r / sig
    g = np.zeros(r.shape + (4, 4))
    g[..., 0, 0] = -(1 - f)
    g[..., 0, 1] = g[..., 1, 0] = f * r
    g[..., 0, 3] = g[..., 3, 0] = -a * f * s2
    g[..., 1, 1] = (1 + f) * r * r
    g[..., 1, 3] = g[..., 3, 1] = -a * s2 * (1 + f) * r
    g[..., 2, 2] = sig * dth * dth
    g[..., 3, 3] = s2 * (sig + a * a * s2 * (1 + f))
    return g


def _fm_torus(r, th, a, r_in, r_max, gam):
    """Fishbone-Moncrief torus (constant l = u^t u_phi): density (max 1), internal energy and the
    Boyer-Lindquist angular velocity.  With l constant the relativistic Euler equation integrates to
    ln h = -ln(-u_t) - l Omega + ln(1 + l Omega) + const; Omega solves
    l g_pp Omega^2 + (2 l g_tp + g_pp) Omega + l g_tt + g_tp = 0 (the BL t-phi block)."""
    def blk(rr, tt):
        s2 = np.sin(tt) ** 2
        sig = rr * rr + a * a * np.cos(tt) ** 2
        gtt = -(1 - 2 * rr / sig)
        gtp = -2 * a * rr * s2 / sig
        gpp = (rr * rr + a * a + 2 * rr * a * a * s2 / sig) * s2
        return gtt, gtp, gpp

    # l of the circular geodesic (Keplerian) at r_max in the equator: Omega_K = 1/(r^1.5 + a)
    gtt, gtp, gpp = blk(np.array(r_max), np.array(np.pi / 2))
    om_k = 1.0 / (r_max ** 1.5 + a)
    ut = 1.0 / np.sqrt(-(gtt + 2 * gtp * om_k + gpp * om_k ** 2))
    l = float(ut * ut * (gtp + gpp * om_k))

    def lnh_raw(rr, tt):
        gtt, gtp, gpp = blk(rr, tt)
        A, B, C = l * gpp, 2 * l * gtp + gpp, l * gtt + gtp
        disc = np.sqrt(np.maximum(B * B - 4 * A * C, 0.0))
        om = (-B + disc) / (2 * A)
        norm = -(gtt + 2 * gtp * om + gpp * om * om)
        ok = norm > 0
        ut = 1.0 / np.sqrt(np.where(ok, norm, 1.0))
        u_t = ut * (gtt + gtp * om)
        val = -np.log(np.where(ok & (u_t < 0), -u_t, 1.0)) - l * om + np.log(np.abs(1 + l * om))
        return np.where(ok & (u_t < 0), val, -np.inf), om, ut

    ref, _, _ = lnh_raw(np.array(r_in), np.array(np.pi / 2))
    lnh, om, ut = lnh_raw(r, th)
    lnh = lnh - ref
    inside = (lnh > 0) & (r >= r_in)
    h = np.exp(np.where(inside, lnh, 0.0))
    # polytrope p = kappa rho^gam: p/rho = (h - 1)(gam - 1)/gam; density normalised to max 1
    rho = np.where(inside, ((h - 1) * (gam - 1) / gam) ** (1 / (gam - 1)), 0.0)
    if not rho.max() > 0:
        raise ValueError("no Fishbone-Moncrief torus for a=%g, r_in=%g, r_max=%g on this grid" % (a, r_in, r_max))
    rho = rho / rho.max()
    u = np.where(inside, (h - 1) / gam * rho, 0.0)   # u = p / (gam - 1)
    return rho, u, np.where(inside, om, 0.0), np.where(inside, ut, 0.0), inside


def r_isco(a):
    """Innermost stable circular orbit (Bardeen, Press & Teukolsky 1972), prograde for a > 0,
    retrograde for a < 0 (M = 1)."""
    z1 = 1 + (1 - a * a) ** (1 / 3) * ((1 + a) ** (1 / 3) + (1 - a) ** (1 / 3))
    z2 = math.sqrt(3 * a * a + z1 * z1)
    return 3 + z2 - math.copysign(math.sqrt((3 - z1) * (3 + z1 + 2 * z2)), a if a != 0 else 1.0)


def torus(*, a=0.9375, n1=256, n2=128, n3=1, r_out=40.0, hslope=0.3, r_in=None, r_max=None, beta_min=100.0,
          pert=0.1, seed=1, m_bh_msun=4.14e6, M_unit=1e18, R_high=20.0, R_low=1.0, dtype=np.float64,
          turb_sigma=0.0, turb_slope=-11.0 / 3.0, **over):
    """Synthetic GRMHD-like snapshot: Fishbone-Moncrief torus (r_in, r_max) around a Kerr hole in
    modified Kerr-Schild coordinates, r from the horizon to r_out, with a single poloidal field loop
    (A_phi ~ max(rho - 0.2, 0)) normalised to min beta = beta_min, atmosphere floors rho = 1e-5 r^-1.5,
    u = 1e-7 r^-2.5, and seeded lognormal perturbations of rho and u (exp(pert N(0,1) - pert^2/2) per
    zone).  With turb_sigma > 0 (3-D grids) a Gaussian random field with power spectrum
    P(k) ~ k^turb_slope (k^-11/3: the 3-D form of a k^-5/3 spectrum) and standard deviation turb_sigma
    multiplies rho and u as exp(delta - sigma^2/2)."""
    gam = GAM
    if r_in is None:   # r_in = 6, r_max = 12 (section 4.3 stand-in) moved outside the ISCO when needed
        r_in = max(6.0, math.ceil(r_isco(a)) + 1.0)
    if r_max is None:
        r_max = max(12.0, 2.0 * r_in)
    rh = 1.0 + math.sqrt(1.0 - a * a)
    g = _grid(n1, n2, n3, math.log(rh), math.log(r_out))
    X1, X2, X3 = _zone_centres(g)
    r = np.exp(X1)
    th = math.pi * X2 + 0.5 * (1 - hslope) * np.sin(2 * math.pi * X2)
    dth = math.pi * (1 + (1 - hslope) * np.cos(2 * math.pi * X2))
    rho, uu, om, ut, inside = _fm_torus(r, th, a, r_in, r_max, gam)
    rng = np.random.default_rng(seed)
    # velocities: torus u^t (1, 0, 0, Omega) (BL = KS components when u^r = 0); normal-observer
    # velocity U^i = u^i - u^t g^{ti}/g^{tt}; KS g^{tr}/g^{tt} = -2r/(Sigma + 2r), g^{tphi} = 0
    sig = r * r + a * a * np.cos(th) ** 2
    U1 = np.where(inside, ut * 2 * r / (sig + 2 * r) / r, 0.0)
    U3 = np.where(inside, ut * om, 0.0)
    # atmosphere at rest with respect to normal observers
    rho_fl, u_fl = 1e-5 * r ** -1.5, 1e-7 * r ** -2.5
    rho = np.maximum(rho, rho_fl)
    uu = np.maximum(uu, u_fl)
    # field from A_phi (zone centres, centred differences in x1, x2): B^1 = -d2 A / sqrt(-g), B^2 = d1 A / sqrt(-g)
    shape = (n1, n2, n3)
    Aphi = np.maximum(rho.reshape(shape) - 0.2, 0.0)
    dA1 = np.gradient(Aphi, g["dx1"], axis=0)
    dA2 = np.gradient(Aphi, g["dx2"], axis=1)
    sqrtg = (sig * np.sin(th) * r * dth).reshape(shape)
    B1 = (-dA2 / sqrtg).ravel()
    B2 = (dA1 / sqrtg).ravel()
    B3 = np.zeros_like(B1)
    # fluid-frame b^2 for the normalisation
    G = _ks_mks_metric(r, th, dth, a)
    Gi = np.linalg.inv(G)
    alpha = 1 / np.sqrt(-Gi[:, 0, 0])
    Ut = np.stack([np.zeros_like(r), U1, np.zeros_like(r), U3], axis=1)
    qq = np.einsum("ni,nij,nj->n", Ut[:, 1:], G[:, 1:, 1:], Ut[:, 1:])
    gamma = np.sqrt(1 + qq)
    ucon = np.stack([gamma / alpha, U1 - gamma * alpha * Gi[:, 0, 1], np.zeros_like(r), U3 - gamma * alpha * Gi[:, 0, 3]], 1)
    ucov = np.einsum("nij,nj->ni", G, ucon)
    Bv = np.stack([np.zeros_like(r), B1, B2, B3], 1)
    bt = np.einsum("ni,ni->n", Bv, ucov)
    bcon = (Bv + bt[:, None] * ucon) / ucon[:, :1]
    bcon[:, 0] = bt
    bsq = np.einsum("ni,nij,nj->n", bcon, G, bcon)
    beta = np.where(bsq > 0, (gam - 1) * uu / (0.5 * np.maximum(bsq, 1e-300)), np.inf)
    sel = inside & (rho > 0.2)
    norm = math.sqrt(beta[sel].min() / beta_min) if sel.any() else 1.0
    B1 *= norm
    B2 *= norm
    # perturbations
    fac = np.exp(pert * rng.standard_normal(r.size) - 0.5 * pert * pert)
    rho = rho * fac
    uu = uu * np.exp(pert * rng.standard_normal(r.size) - 0.5 * pert * pert)
    if turb_sigma > 0 and n3 > 1:
        kx = np.fft.fftfreq(n1)[:, None, None]
        ky = np.fft.fftfreq(n2)[None, :, None]
        kz = np.fft.fftfreq(n3)[None, None, :]
        k = np.sqrt(kx * kx + ky * ky + kz * kz)
        amp = np.where(k > 0, np.where(k > 0, k, 1.0) ** (turb_slope / 2.0), 0.0)
        noise = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        delta = np.real(np.fft.ifftn(noise * amp))
        delta *= turb_sigma / delta.std()
        d = delta.ravel()
        rho = rho * np.exp(d - 0.5 * turb_sigma ** 2)
        uu = uu * np.exp(d - 0.5 * turb_sigma ** 2)
    prim = np.stack([rho, uu, B1, B2, B3, U1, np.zeros_like(r), U3]).astype(dtype)
    g["prim"] = prim
    params = base_params(a=a, mass=1.0, hslope=hslope, L_unit=length_unit(m_bh_msun), M_unit=M_unit,
                         R_high=R_high, R_low=R_low, w_min=1e20, scatter=1, bias_mode=2, bias_p0=96e4,
                         bias_max=1e5, n_sc_max=3, dh=0.05)
    params.update(over)
    return params, g


def torus3d(**over):
    """3-D snapshot stand-in: a = 0.5, 288 x 128 x 128, FP32 fields, torus x lognormal turbulence
    (sigma 0.1, P(k) ~ k^-11/3), 6 inclination bins, mixed precision intended."""
    kw = dict(a=0.5, n1=288, n2=128, n3=128, dtype=np.float32, turb_sigma=0.1, n_incl=6)
    kw.update(over)
    return torus(**kw)


def survey(n_models=64, seed=1):
    """Batched parameter survey: models drawn (seeded) from spin {-0.94,-0.5,0,0.5,0.94} x
    R_high {1,10,40,160} x accretion-rate scale {0.5,1,2,4} (M_unit = 5e17 g x scale), grids 128x64,
    192x96 or 256x128, N_s log-uniform in [1e5, 1e7].  Returns a list of (params, grid, N_s)."""
    rng = np.random.default_rng(seed)
    spins = [-0.94, -0.5, 0.0, 0.5, 0.94]
    rhs = [1.0, 10.0, 40.0, 160.0]
    scales = [0.5, 1.0, 2.0, 4.0]
    grids = [(128, 64), (192, 96), (256, 128)]
    out = []
    for i in range(n_models):
        a = spins[rng.integers(len(spins))]
        rh = rhs[rng.integers(len(rhs))]
        sc = scales[rng.integers(len(scales))]
        n1, n2 = grids[rng.integers(len(grids))]
        ns = float(10 ** rng.uniform(5, 7))
        p, g = torus(a=a, n1=n1, n2=n2, R_high=rh, M_unit=5e17 * sc, seed=seed * 1000 + i)
        out.append((p, g, ns))
    return out
