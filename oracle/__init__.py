"""Plain FP64 CPU oracle for the GPUmonty Monte Carlo hot path (arXiv 2602.13198).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product path (the CUDA library and its binding) never imports, links or runs it.

The arithmetic lives in ``mc_oracle.cpp`` (C++17, FP64, no code shared with the
CUDA path).  This module compiles it with g++ on first use (or via :func:`build`) and
exposes thin ctypes wrappers.  Parity status per function is stated in the C++ header
comment; every function cites the section of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mc_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "libmc_oracle.so")
_lock = threading.Lock()
_lib = None


class Params(C.Structure):
    """Mirror of ``or_params`` (oracle's own parameter struct)."""
    _fields_ = [
        ("a", C.c_double), ("mass", C.c_double), ("hslope", C.c_double),
        ("L_unit", C.c_double), ("M_unit", C.c_double),
        ("R_high", C.c_double), ("R_low", C.c_double), ("gam", C.c_double),
        ("thetae_min", C.c_double), ("thetae_max", C.c_double),
        ("nu_min", C.c_double), ("nu_max", C.c_double),
        ("w_min", C.c_double), ("n_s", C.c_double),
        ("eps_geo", C.c_double), ("verlet_tol", C.c_double),
        ("r_record", C.c_double), ("dh", C.c_double), ("bias_p0", C.c_double),
        ("lnu_lo", C.c_double), ("lnu_hi", C.c_double),
        ("roulette_w", C.c_double), ("roulette_p", C.c_double), ("bias_max", C.c_double),
        ("kappa", C.c_double), ("bias_target", C.c_double),
        ("max_steps", C.c_int64),
        ("n_nu", C.c_int32), ("verlet_maxit", C.c_int32), ("bias_mode", C.c_int32),
        ("n_sc_max", C.c_int32), ("n_bins", C.c_int32), ("n_incl", C.c_int32),
        ("k2_mode", C.c_int32), ("scatter", C.c_int32), ("brems", C.c_int32),
    ]


class Grid(C.Structure):
    _fields_ = [
        ("n1", C.c_int32), ("n2", C.c_int32), ("n3", C.c_int32), ("pad", C.c_int32),
        ("x1_0", C.c_double), ("dx1", C.c_double), ("x2_0", C.c_double),
        ("dx2", C.c_double), ("x3_0", C.c_double), ("dx3", C.c_double),
        ("prim", C.POINTER(C.c_double)),
    ]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "n_emit", "n_child", "n_rec", "n_abs", "n_capt", "n_maxst",
        "n_steps", "n_iters", "n_nonconv", "n_roul_surv", "n_rej_cap", "n_events")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


LOG_DTYPE = np.dtype([
    ("id", np.uint64), ("gen", np.int32), ("status", np.int32),
    ("X", np.float64, 4), ("K", np.float64, 4), ("w", np.float64),
    ("nsteps", np.int64), ("nev", np.int32), ("pad", np.int32)])


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (g++, -O2, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + ".tmp%d" % os.getpid()
            cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
            subprocess.check_call(cmd)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P, D, I64, U64, U32 = C.POINTER, C.c_double, C.c_int64, C.c_uint64, C.c_uint32
        PD = P(D)
        L.or_philox.argtypes = [P(U32), P(U32), P(U32)]
        L.or_uniforms.argtypes = [U64, U64, U32, I64, PD]
        L.or_child_stream.argtypes = [U64, U32]
        L.or_child_stream.restype = U64
        L.or_gauss_legendre.argtypes = [C.c_int, D, D, PD, PD]
        L.or_gcov.argtypes = [P(Params), PD, PD]
        L.or_sqrtmg.argtypes = [P(Params), PD]
        L.or_sqrtmg.restype = D
        L.or_christoffel.argtypes = [P(Params), PD, PD]
        L.or_geodesic.argtypes = [P(Params), PD, PD, D, D, I64, PD, PD, PD, P(I64)]
        L.or_geodesic.restype = I64
        L.or_jnu.argtypes = [P(Params), D, D, D, D, D]
        L.or_jnu.restype = D
        L.or_bnu.argtypes = [D, D]
        L.or_bnu.restype = D
        L.or_K2.argtypes = [P(Params), D]
        L.or_K2.restype = D
        L.or_Fang.argtypes = [D]
        L.or_Fang.restype = D
        L.or_jnu_angint.argtypes = [P(Params), D, D, D, D]
        L.or_jnu_angint.restype = D
        L.or_sigma_kn.argtypes = [D]
        L.or_sigma_kn.restype = D
        L.or_sigma_hot_quad.argtypes = [D, D]
        L.or_sigma_hot_quad.restype = D
        L.or_sigma_hot_table.argtypes = [D, D]
        L.or_sigma_hot_table.restype = D
        L.or_sample_mj.argtypes = [D, U64, U64, I64, PD]
        L.or_compton.argtypes = [D, D, U64, U64, I64, PD, PD]
        L.or_fluid.argtypes = [C.c_void_p, PD, PD]
        L.or_fluid_from_prims.argtypes = [P(Params), PD, PD, PD]
        L.or_tetrad.argtypes = [P(Params), PD, PD, C.c_int, PD]
        L.or_create.argtypes = [P(Params), P(Grid)]
        L.or_create.restype = C.c_void_p
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_prepare.argtypes = [C.c_void_p, D, U64]
        L.or_total.argtypes = [C.c_void_p]
        L.or_total.restype = I64
        L.or_nzones.argtypes = [C.c_void_p]
        L.or_nzones.restype = I64
        L.or_get_zone.argtypes = [C.c_void_p, P(I64), PD, PD, PD]
        L.or_get_weights.argtypes = [C.c_void_p, PD]
        L.or_emit.argtypes = [C.c_void_p, I64, I64, PD, PD, PD]
        L.or_run.argtypes = [C.c_void_p, I64, I64, P(I64), I64, PD, P(Stats), C.c_void_p, I64, P(I64), C.c_int]
        L.or_get_bias_scales.argtypes = [C.c_void_p, PD, C.c_int]
        L.or_sigma_hot_kappa.argtypes = [D, D, D]
        L.or_sigma_hot_kappa.restype = D
        L.or_sample_kappa.argtypes = [D, D, U64, U64, I64, PD]
        L.or_compton_kappa.argtypes = [D, D, D, U64, U64, I64, PD, PD]
        L.or_F_sync.argtypes = [D]
        L.or_F_sync.restype = D
        L.or_jnu_kappa.argtypes = [P(Params), D, D, D, D, D]
        L.or_jnu_kappa.restype = D
        L.or_nu_alpha_kappa.argtypes = [P(Params), D, D, D, D, D]
        L.or_nu_alpha_kappa.restype = D
        L.or_brems_q.argtypes = [D, D]
        L.or_brems_q.restype = D
        L.or_brems_angint.argtypes = [P(Params), D, D, D]
        L.or_brems_angint.restype = D
        L.or_brems_nu_alpha.argtypes = [P(Params), D, D, D]
        L.or_brems_nu_alpha.restype = D
        _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def params_from(cfg: dict) -> Params:
    """Build the oracle's parameter struct from a plain model dictionary."""
    p = Params()
    for name, _ in Params._fields_:
        setattr(p, name, cfg[name])
    return p


# ----------------------------------------------------------------- scalar helpers
def philox(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    L.or_philox(c, k, o)
    return [int(v) for v in o]


def uniforms(seed, stream, n, start=0):
    out = np.empty(n)
    lib().or_uniforms(seed, stream, start, n, _pd(out))
    return out


def child_stream(parent, ev):
    return int(lib().or_child_stream(parent, ev))


def gauss_legendre(n, a=-1.0, b=1.0):
    x = np.empty(n)
    w = np.empty(n)
    lib().or_gauss_legendre(n, a, b, _pd(x), _pd(w))
    return x, w


def gcov(cfg, X):
    p = params_from(cfg)
    X = np.ascontiguousarray(X, dtype=np.float64)
    g = np.empty(16)
    lib().or_gcov(C.byref(p), _pd(X), _pd(g))
    return g.reshape(4, 4)


def sqrtmg(cfg, X):
    p = params_from(cfg)
    X = np.ascontiguousarray(X, dtype=np.float64)
    return lib().or_sqrtmg(C.byref(p), _pd(X))


def christoffel(cfg, X):
    p = params_from(cfg)
    X = np.ascontiguousarray(X, dtype=np.float64)
    G = np.empty(64)
    lib().or_christoffel(C.byref(p), _pd(X), _pd(G))
    return G.reshape(4, 4, 4)


def geodesic(cfg, X0, K0, r_in, r_out, max_steps=100000):
    p = params_from(cfg)
    X0 = np.ascontiguousarray(X0, dtype=np.float64)
    K0 = np.ascontiguousarray(K0, dtype=np.float64)
    Xe = np.empty(4)
    Ke = np.empty(4)
    mn = np.empty(1)
    its = C.c_int64(0)
    n = lib().or_geodesic(C.byref(p), _pd(X0), _pd(K0), r_in, r_out, max_steps, _pd(Xe), _pd(Ke), _pd(mn), C.byref(its))
    return {"X": Xe, "K": Ke, "nsteps": int(n), "max_null": float(mn[0]), "iters": int(its.value)}


def fluid_from_prims(cfg, X, prim):
    """Fluid state at X from the primitives (rho, u, B^1..3, U^1..3): dict with ne, thetae, B [G],
    bsq, ucon, ucov, bcon, bcov."""
    p = params_from(cfg)
    X = np.ascontiguousarray(X, dtype=np.float64)
    pr = np.ascontiguousarray(prim, dtype=np.float64)
    out = np.empty(20)
    lib().or_fluid_from_prims(C.byref(p), _pd(X), _pd(pr), _pd(out))
    return {"ne": out[0], "thetae": out[1], "B": out[2], "bsq": out[3], "ucon": out[4:8].copy(),
            "ucov": out[8:12].copy(), "bcon": out[12:16].copy(), "bcov": out[16:20].copy()}


def tetrad(cfg, X, prim, kind):
    """Plasma-frame tetrad e[a, mu] at X for the primitives: kind "emission" or "scatter"."""
    p = params_from(cfg)
    X = np.ascontiguousarray(X, dtype=np.float64)
    pr = np.ascontiguousarray(prim, dtype=np.float64)
    e = np.empty(16)
    lib().or_tetrad(C.byref(p), _pd(X), _pd(pr), 0 if kind == "emission" else 1, _pd(e))
    return e.reshape(4, 4)


def jnu(cfg, nu, ne, thetae, B, costh):
    p = params_from(cfg)
    return lib().or_jnu(C.byref(p), nu, ne, thetae, B, costh)


def bnu(nu, thetae):
    return lib().or_bnu(nu, thetae)


def K2(cfg, thetae):
    p = params_from(cfg)
    return lib().or_K2(C.byref(p), thetae)


def Fang(K):
    return lib().or_Fang(K)


def jnu_angint(cfg, nu, ne, thetae, B):
    p = params_from(cfg)
    return lib().or_jnu_angint(C.byref(p), nu, ne, thetae, B)


def sigma_hot_kappa(kappa, w, eps):
    return lib().or_sigma_hot_kappa(kappa, w, eps)


def sample_kappa(kappa, w, n, seed=1, stream=0):
    out = np.empty(n)
    lib().or_sample_kappa(kappa, w, seed, stream, n, _pd(out))
    return out


def compton_kappa(kappa, thetae, eps, n, seed=1, stream0=0):
    e = np.empty(n)
    mu = np.empty(n)
    lib().or_compton_kappa(kappa, thetae, eps, seed, stream0, n, _pd(e), _pd(mu))
    return e, mu


def F_sync(x):
    return lib().or_F_sync(x)


def jnu_kappa(cfg, nu, ne, thetae, B, costh):
    p = params_from(cfg)
    return lib().or_jnu_kappa(C.byref(p), nu, ne, thetae, B, costh)


def nu_alpha_kappa(cfg, nu, ne, thetae, B, costh):
    p = params_from(cfg)
    return lib().or_nu_alpha_kappa(C.byref(p), nu, ne, thetae, B, costh)


def brems_q(ne, thetae):
    return lib().or_brems_q(ne, thetae)


def brems_angint(cfg, nu, ne, thetae):
    p = params_from(cfg)
    return lib().or_brems_angint(C.byref(p), nu, ne, thetae)


def brems_nu_alpha(cfg, nu, ne, thetae):
    p = params_from(cfg)
    return lib().or_brems_nu_alpha(C.byref(p), nu, ne, thetae)


def sigma_kn(e):
    return lib().or_sigma_kn(e)


def sigma_hot_quad(thetae, eps):
    return lib().or_sigma_hot_quad(thetae, eps)


def sigma_hot_table(thetae, eps):
    return lib().or_sigma_hot_table(thetae, eps)


def sample_mj(thetae, n, seed=1, stream=0):
    out = np.empty(n)
    lib().or_sample_mj(thetae, seed, stream, n, _pd(out))
    return out


def compton(thetae, eps, n, seed=1, stream0=0):
    e = np.empty(n)
    d = np.empty((n, 3))
    lib().or_compton(thetae, eps, seed, stream0, n, _pd(e), _pd(d))
    return e, d


# ----------------------------------------------------------------- full model
class Model:
    """One model: parameters + grid.  ``prepare`` computes weights and zone counts,
    ``run`` transports primaries (and all their descendants)."""

    def __init__(self, cfg: dict, grid: dict):
        self.cfg = dict(cfg)
        self._p = params_from(cfg)
        prim = np.ascontiguousarray(grid["prim"], dtype=np.float64)
        self._prim = prim
        g = Grid()
        g.n1, g.n2, g.n3 = grid["n1"], grid["n2"], grid["n3"]
        for k in ("x1_0", "dx1", "x2_0", "dx2", "x3_0", "dx3"):
            setattr(g, k, grid[k])
        g.prim = _pd(prim)
        self._g = g
        self._h = lib().or_create(C.byref(self._p), C.byref(g))
        self.nz = int(lib().or_nzones(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def prepare(self, n_s, seed):
        lib().or_prepare(self._h, float(n_s), int(seed))
        return int(lib().or_total(self._h))

    @property
    def total(self):
        return int(lib().or_total(self._h))

    def zones(self):
        n = self.nz
        counts = np.empty(n, dtype=np.int64)
        nbar = np.empty(n)
        gmax = np.empty(n)
        vol = np.empty(n)
        lib().or_get_zone(self._h, counts.ctypes.data_as(C.POINTER(C.c_int64)), _pd(nbar), _pd(gmax), _pd(vol))
        return {"counts": counts, "nbar": nbar, "gmax": gmax, "vol": vol}

    def lnw(self):
        out = np.empty(self.cfg["n_nu"])
        lib().or_get_weights(self._h, _pd(out))
        return out

    def emit(self, uid0=0, n=None):
        """Birth states (X, K, w) of primaries [uid0, uid0 + n) after prepare: emission only."""
        if n is None:
            n = self.total - uid0
        X, K, w = np.empty((n, 4)), np.empty((n, 4)), np.empty(n)
        lib().or_emit(self._h, int(uid0), int(n), _pd(X), _pd(K), _pd(w))
        return X, K, w

    def fluid(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        out = np.empty(12)
        lib().or_fluid(self._h, _pd(X), _pd(out))
        return {"ne": out[0], "thetae": out[1], "B": out[2], "plasma": bool(out[3]),
                "ucon": out[4:8].copy(), "bcon": out[8:12].copy()}

    def bias_scales(self):
        """Bias scale per scattering generation of the last range run."""
        out = np.empty(int(self.cfg["n_sc_max"]) + 1)
        lib().or_get_bias_scales(self._h, _pd(out), len(out))
        return out

    def run(self, uid0=0, uid1=None, uids=None, nthreads=None, log=False, log_cap=None):
        c = self.cfg
        if uid1 is None:
            uid1 = self.total
        if nthreads is None:
            nthreads = os.cpu_count() or 1
        spec = np.zeros((c["n_incl"], c["n_bins"], 3))
        st = Stats()
        ul = None
        nu = 0
        if uids is not None:
            ul = np.ascontiguousarray(uids, dtype=np.int64)
            nu = len(ul)
        logbuf = None
        logn = C.c_int64(0)
        if log:
            cap = log_cap if log_cap is not None else max(16, 64 * ((nu if ul is not None else uid1 - uid0) + 1))
            logbuf = np.zeros(cap, dtype=LOG_DTYPE)
        lib().or_run(self._h, int(uid0), int(uid1),
                     ul.ctypes.data_as(C.POINTER(C.c_int64)) if ul is not None else None, nu,
                     _pd(spec), C.byref(st),
                     logbuf.ctypes.data if logbuf is not None else None,
                     len(logbuf) if logbuf is not None else 0, C.byref(logn), int(nthreads))
        out = {"spec": spec, "stats": st.as_dict()}
        if log:
            out["log"] = logbuf[: logn.value].copy()
        return out
