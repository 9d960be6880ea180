"""Thin ctypes binding of the C ABI in ``include/mc.h`` (argument marshalling only).

Every step of the hot path runs in the CUDA library ``libmcgb.so``; this module only
fills the parameter structs, hands PyTorch's caching allocator to the library, and
copies results out.  Importing works without a GPU; creating a :class:`Model` without
one raises :class:`MCError` (``MC_ERR_NO_DEVICE``).  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmcgb.so")

MC_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "NO_DEVICE", -3: "OOM", -4: "TIMEOUT", -5: "QUEUE_OVERFLOW",
          -6: "NAN_INPUT", -7: "SIZE", -8: "STATE", -9: "CUDA"}
PREC = {"fp64": 0, "mixed": 1, "split": 2}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class MCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class ModelParams(C.Structure):
    _fields_ = [
        ("a", C.c_double), ("mass", C.c_double), ("hslope", C.c_double),
        ("L_unit", C.c_double), ("M_unit", C.c_double),
        ("R_high", C.c_double), ("R_low", C.c_double), ("gam", C.c_double),
        ("thetae_min", C.c_double), ("thetae_max", C.c_double),
        ("nu_min", C.c_double), ("nu_max", C.c_double), ("w_min", C.c_double), ("n_s", C.c_double),
        ("eps_geo", C.c_double), ("verlet_tol", C.c_double), ("r_record", C.c_double), ("dh", C.c_double),
        ("bias_p0", C.c_double), ("lnu_lo", C.c_double), ("lnu_hi", C.c_double),
        ("roulette_w", C.c_double), ("roulette_p", C.c_double), ("bias_max", C.c_double),
        ("kappa", C.c_double), ("bias_target", C.c_double),
        ("max_steps", C.c_int64),
        ("n_nu", C.c_int32), ("verlet_maxit", C.c_int32), ("bias_mode", C.c_int32), ("n_sc_max", C.c_int32),
        ("n_bins", C.c_int32), ("n_incl", C.c_int32), ("k2_mode", C.c_int32), ("scatter", C.c_int32),
        ("precision", C.c_int32), ("surrogate", C.c_int32), ("block", C.c_int32), ("ctas_per_sm", C.c_int32),
        ("device", C.c_int32), ("brems", C.c_int32),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
    ]


class GridDesc(C.Structure):
    _fields_ = [
        ("n1", C.c_int32), ("n2", C.c_int32), ("n3", C.c_int32), ("dtype", C.c_int32),
        ("x1_0", C.c_double), ("dx1", C.c_double), ("x2_0", C.c_double), ("dx2", C.c_double),
        ("x3_0", C.c_double), ("dx3", C.c_double),
        ("location", C.c_int32), ("pad0", C.c_int32), ("prim", C.c_void_p),
    ]


INT_STATS = ("n_emit", "n_child", "n_rec", "n_abs", "n_capt", "n_maxst", "n_steps", "n_iters",
             "n_nonconv", "n_roul_surv", "n_rej_cap", "n_events", "n_total", "err_flags", "transport_launches")


class RunStats(C.Structure):
    _fields_ = ([(n, C.c_int64) for n in INT_STATS] + [("transport_ms", C.c_double), ("generate_ms", C.c_double)] +
                [("n_steps_grid", C.c_int64), ("n_iters_grid", C.c_int64)] +
                [("init_ms", C.c_double), ("grid_ms", C.c_double), ("free_ms", C.c_double)] +
                [("batch_min_blocks", C.c_int32), ("batch_ctas", C.c_int32), ("batch_graph", C.c_int32),
                 ("pad0", C.c_int32)])

    def as_dict(self):
        d = {}
        for n, t in self._fields_:
            v = getattr(self, n)
            if n != "pad0":
                d[n] = float(v) if t is C.c_double else int(v)
        return d


LOG_DTYPE = np.dtype([
    ("id", np.uint64), ("gen", np.int32), ("status", np.int32),
    ("X", np.float64, 4), ("K", np.float64, 4), ("w", np.float64),
    ("nsteps", np.int64), ("nev", np.int32), ("pad", np.int32)])

_lib = None


def lib():
    """Loads libmcgb.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MCError(-9, "CUDA library %s missing: run paper_2602_13198_gb300.build.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, i64, u64, sz, dp = C.c_void_p, C.c_int64, C.c_uint64, C.c_size_t, C.POINTER(C.c_double)
        L.mc_init_model.argtypes = [C.POINTER(vp), C.POINTER(ModelParams)]
        L.mc_set_grid.argtypes = [vp, C.POINTER(GridDesc)]
        L.mc_run.argtypes = [vp, C.c_double, u64, i64, i64, vp, C.POINTER(RunStats)]
        L.mc_get_spectrum.argtypes = [vp, dp, dp, dp, sz]
        L.mc_get_spectrum_sums.argtypes = [vp, dp, sz]
        L.mc_get_zone_counts.argtypes = [vp, C.POINTER(i64), sz]
        L.mc_trace.argtypes = [vp, C.c_double, u64, C.POINTER(i64), sz, vp, sz, C.POINTER(sz), vp]
        L.mc_free.argtypes = [vp]
        L.mc_free.restype = None
        L.mc_last_error.argtypes = [vp]
        L.mc_last_error.restype = C.c_char_p
        L.mc_version.restype = C.c_char_p
        L.mc_fma_peak.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double)]
        L.mc_fma_peak.restype = C.c_int
        L.mc_get_bias_scales.argtypes = [vp, C.POINTER(C.c_double), C.c_int]
        L.mc_get_bias_scales.restype = C.c_int
        L.mc_selftest_math.argtypes = [C.c_int, vp, vp, vp, C.c_int64]
        L.mc_selftest_math.restype = C.c_int
        L.mc_run_batch.argtypes = [C.POINTER(vp), C.c_int, dp, C.POINTER(u64), C.c_int, vp, C.POINTER(RunStats)]
        L.mc_run_batch.restype = C.c_int
        L.mc_zone_counts_noalloc.argtypes = [vp, C.c_double, u64, vp, vp, vp, vp]
        L.mc_zone_counts_noalloc.restype = C.c_int
        L.mc_set_wait_limit.argtypes = [vp, C.c_double]
        L.mc_set_wait_limit.restype = C.c_int
        fp = C.POINTER(C.c_float)
        L.mc_surrogate_train.argtypes = [vp, i64, i64, i64, C.c_double, u64, dp]
        L.mc_surrogate_set_weights.argtypes = [vp, fp]
        L.mc_surrogate_get_weights.argtypes = [vp, fp]
        L.mc_surrogate_grad.argtypes = [vp, fp, fp, fp, fp, i64, fp, dp]
        L.mc_surrogate_infer.argtypes = [vp, fp, fp, i64, C.c_int]
        for f in ("mc_surrogate_train", "mc_surrogate_set_weights", "mc_surrogate_get_weights",
                  "mc_surrogate_grad", "mc_surrogate_infer"):
            getattr(L, f).restype = C.c_int
        for f in ("mc_init_model", "mc_set_grid", "mc_run", "mc_get_spectrum", "mc_get_spectrum_sums",
                  "mc_get_zone_counts", "mc_trace"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _torch_allocator():
    """Device allocator callbacks backed by PyTorch's caching allocator."""
    import torch

    def _alloc(nbytes, user):
        dev = torch.cuda.current_device()
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev))

    def _free(ptr, user):
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)
    return ALLOC_FN(_alloc), FREE_FN(_free)


class Model:
    """One model context: ``Model(params, device=0)`` then ``set_grid`` and ``run``.

    ``precision="fp64"`` runs every step in FP64.  ``precision="mixed"`` runs the geodesic in
    double-float on the FP32 pipes (FP64-level accuracy) and the plasma coefficients, optical
    depths and weights in FP32; ``precision="split"`` runs the geodesic in FP64 and the rest in
    FP32 (see ``precision`` in include/mc.h); ``surrogate=True`` (mixed or split) takes K2,
    sigma_h and the emissivity shape from the tensor-core network."""

    def __init__(self, params: dict, device: int = 0, precision: str = "fp64", use_torch_allocator: bool = True,
                 block: int = 0, ctas_per_sm: int = 0, surrogate: bool = False):
        L = lib()
        p = ModelParams()
        for name, _ in ModelParams._fields_:
            if name in params and name not in ("alloc", "free", "alloc_user"):
                setattr(p, name, params[name])
        p.precision = PREC[precision] if isinstance(precision, str) else int(precision)
        p.surrogate = 1 if surrogate else 0
        p.block = block
        p.ctas_per_sm = ctas_per_sm
        p.device = device
        self._cb = None
        if use_torch_allocator:
            import torch
            torch.cuda.set_device(device)
            self._cb = _torch_allocator()
            p.alloc, p.free = self._cb
        self.params = dict(params)
        self._p = p
        h = C.c_void_p()
        rc = L.mc_init_model(C.byref(h), C.byref(p))
        if rc != MC_OK:
            raise MCError(rc, L.mc_last_error(None).decode())
        self._h = h
        self.n_incl = int(params["n_incl"])
        self.n_bins = int(params["n_bins"])
        self.n_sc_max = int(params["n_sc_max"])
        self.nz = 0

    def close(self):
        if getattr(self, "_h", None):
            lib().mc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != MC_OK:
            raise MCError(rc, lib().mc_last_error(self._h).decode())

    def set_grid(self, grid: dict, prim=None):
        """``grid`` from :mod:`synth`; ``prim`` may be a CUDA torch tensor [8, nz] (device copy) or
        None to pass ``grid['prim']`` (a numpy array) from host memory."""
        g = GridDesc()
        g.n1, g.n2, g.n3 = grid["n1"], grid["n2"], grid["n3"]
        for k in ("x1_0", "dx1", "x2_0", "dx2", "x3_0", "dx3"):
            setattr(g, k, grid[k])
        keep = None
        if prim is not None and hasattr(prim, "is_cuda") and prim.is_cuda:
            keep = prim.contiguous()
            g.dtype = 1 if str(keep.dtype) == "torch.float32" else 0
            g.location = 1
            g.prim = keep.data_ptr()
        else:
            arr = grid["prim"] if prim is None else prim
            keep = np.ascontiguousarray(arr)
            if keep.dtype == np.float32:
                g.dtype = 1
            else:
                keep = np.ascontiguousarray(keep, dtype=np.float64)
                g.dtype = 0
            g.location = 0
            g.prim = keep.ctypes.data
        self._check(lib().mc_set_grid(self._h, C.byref(g)))
        self.nz = g.n1 * g.n2 * g.n3

    def run(self, n_s: float, seed: int, shard: int = 0, n_shards: int = 1, stream=None) -> dict:
        st = RunStats()
        s = C.c_void_p(stream) if isinstance(stream, int) else C.c_void_p(getattr(stream, "cuda_stream", 0) or 0)
        self._check(lib().mc_run(self._h, float(n_s), int(seed), int(shard), int(n_shards), s, C.byref(st)))
        return st.as_dict()

    def spectrum(self):
        n = self.n_incl * self.n_bins
        nuL, sig, cnt = np.zeros(n), np.zeros(n), np.zeros(n)
        dp = C.POINTER(C.c_double)
        self._check(lib().mc_get_spectrum(self._h, nuL.ctypes.data_as(dp), sig.ctypes.data_as(dp),
                                          cnt.ctypes.data_as(dp), n))
        sh = (self.n_incl, self.n_bins)
        return nuL.reshape(sh), sig.reshape(sh), cnt.reshape(sh)

    def bias_scales(self):
        """Bias scale per scattering generation of the last run (mc_get_bias_scales)."""
        out = np.zeros(self.n_sc_max + 1)
        self._check(lib().mc_get_bias_scales(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), len(out)))
        return out

    def spectrum_sums(self):
        n = self.n_incl * self.n_bins * 3
        out = np.zeros(n)
        self._check(lib().mc_get_spectrum_sums(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), n))
        return out.reshape(self.n_incl, self.n_bins, 3)

    def zone_counts(self):
        out = np.zeros(self.nz, dtype=np.int64)
        self._check(lib().mc_get_zone_counts(self._h, out.ctypes.data_as(C.POINTER(C.c_int64)), self.nz))
        return out

    def set_wait_limit(self, seconds: float):
        """Limit on each grid-barrier wait of a batch this model leads (mc_set_wait_limit)."""
        self._check(lib().mc_set_wait_limit(self._h, float(seconds)))

    def zone_counts_noalloc(self, n_s: float, seed: int, counts, start, total, stream=None):
        """Zone counts into caller-owned CUDA tensors (int64 [nz], [nz], [1]) with no device
        allocation inside the library (see mc_zone_counts_noalloc in include/mc.h)."""
        s = C.c_void_p(getattr(stream, "cuda_stream", 0) or 0) if stream is not None else C.c_void_p(0)
        self._check(lib().mc_zone_counts_noalloc(self._h, float(n_s), int(seed), C.c_void_p(counts.data_ptr()),
                                                 C.c_void_p(start.data_ptr()), C.c_void_p(total.data_ptr()), s))

    # ---------------------------------------------------------------- coefficient surrogate
    N_WEIGHTS = 4611

    def surrogate_train(self, n_train=1 << 18, steps=8000, batch=4096, lr=3e-3, seed=1) -> float:
        """Trains the surrogate on the GPU (data from the library's own quadratures); returns the
        validation loss (mean squared error in the scaled outputs)."""
        v = C.c_double(0.0)
        self._check(lib().mc_surrogate_train(self._h, int(n_train), int(steps), int(batch), float(lr), int(seed),
                                             C.byref(v)))
        return v.value

    def surrogate_weights(self, w=None):
        fp = C.POINTER(C.c_float)
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.float32)
            self._check(lib().mc_surrogate_set_weights(self._h, w.ctypes.data_as(fp)))
            return w
        out = np.zeros(self.N_WEIGHTS, dtype=np.float32)
        self._check(lib().mc_surrogate_get_weights(self._h, out.ctypes.data_as(fp)))
        return out

    def surrogate_grad(self, w, x, t, mask):
        fp = C.POINTER(C.c_float)
        w = np.ascontiguousarray(w, dtype=np.float32)
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        mask = np.ascontiguousarray(mask, dtype=np.float32)
        g = np.zeros(self.N_WEIGHTS, dtype=np.float32)
        loss = C.c_double(0.0)
        self._check(lib().mc_surrogate_grad(self._h, w.ctypes.data_as(fp), x.ctypes.data_as(fp), t.ctypes.data_as(fp),
                                            mask.ctypes.data_as(fp), len(x), g.ctypes.data_as(fp), C.byref(loss)))
        return g, loss.value

    def surrogate_infer(self, x, tensor_cores=True):
        fp = C.POINTER(C.c_float)
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros_like(x)
        self._check(lib().mc_surrogate_infer(self._h, x.ctypes.data_as(fp), y.ctypes.data_as(fp), len(x),
                                             1 if tensor_cores else 0))
        return y

    def trace(self, n_s: float, seed: int, uids, cap: int | None = None, stream=None):
        u = np.ascontiguousarray(uids, dtype=np.int64)
        if cap is None:
            cap = max(64, 64 * len(u))
        out = np.zeros(cap, dtype=LOG_DTYPE)
        n = C.c_size_t(0)
        s = C.c_void_p(getattr(stream, "cuda_stream", 0) or 0) if stream is not None else C.c_void_p(0)
        self._check(lib().mc_trace(self._h, float(n_s), int(seed), u.ctypes.data_as(C.POINTER(C.c_int64)), len(u),
                                   out.ctypes.data, cap, C.byref(n), s))
        return out[: n.value].copy()


def run_batch(models, n_s, seeds, autotune=True, graph=True, stream=None) -> dict:
    """Runs several models in one persistent launch (mc_run_batch); spectra are read per model."""
    n = len(models)
    hs = (C.c_void_p * n)(*[m._h.value for m in models])
    ns = (C.c_double * n)(*[float(x) for x in n_s])
    sd = (C.c_uint64 * n)(*[int(x) for x in seeds])
    flags = (1 if autotune else 0) | (2 if graph else 0)
    st = RunStats()
    s = C.c_void_p(getattr(stream, "cuda_stream", 0) or 0) if stream is not None else C.c_void_p(0)
    rc = lib().mc_run_batch(hs, n, ns, sd, flags, s, C.byref(st))
    if rc != MC_OK:
        raise MCError(rc, lib().mc_last_error(models[0]._h).decode())
    return st.as_dict()


def fma_peak(device: int = 0, fp64: bool = True) -> float:
    """FP64 (or FP32) FMA-chain throughput of the device in FLOP/s."""
    f = C.c_double(0.0)
    rc = lib().mc_fma_peak(device, 0 if fp64 else 1, C.byref(f))
    if rc != MC_OK:
        raise MCError(rc, lib().mc_last_error(None).decode())
    return f.value


def selftest_math(which: int, x):
    """Test hook: (library implementation, CUDA reference) of special function `which` at x (see
    mc_selftest_math in include/mc.h)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y, ref = np.empty_like(x), np.empty_like(x)
    rc = lib().mc_selftest_math(int(which), x.ctypes.data, y.ctypes.data, ref.ctypes.data, len(x))
    if rc != MC_OK:
        raise MCError(rc, lib().mc_last_error(None).decode())
    return y, ref


def version() -> str:
    return lib().mc_version().decode()


# ------------------------------------------------------------- multi-rank jobs (one process per GPU)
# Superphotons are independent once the weights and zone counts are fixed (section 2.3), so a job
# shards by contiguous uid ranges of its primaries; scattered children stay with their parent's
# rank.  Every rank computes the same weights and counts; the only exchange is one sum-allreduce
# of the spectrum accumulators (and of the counters) at the end.
SUMMED_STATS = ("n_emit", "n_child", "n_rec", "n_abs", "n_capt", "n_maxst", "n_steps", "n_iters", "n_nonconv",
                "n_roul_surv", "n_rej_cap", "n_events", "n_steps_grid", "n_iters_grid")


def shard_bounds(total: int, shard: int, n_shards: int):
    """uid range [u0, u1) of shard `shard` of `n_shards` over `total` primaries: the contiguous
    split mc_run applies (u0 = floor(total * shard / n_shards))."""
    if n_shards < 1 or not 0 <= shard < n_shards:
        raise ValueError("bad shard")
    return (total * shard) // n_shards, (total * (shard + 1)) // n_shards


def _allreduce(arr, dtype, group):
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(arr, dtype=dtype).copy())
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def allreduce_spectrum(sums, group=None):
    """Sum over the ranks of `group` of spectrum accumulators (sum wE, sum (wE)^2, count) in FP64
    (host tensors under gloo, device tensors under NCCL)."""
    return _allreduce(sums, np.float64, group)


def allreduce_stats(stats: dict, group=None) -> dict:
    """Counters of a sharded job: event counts summed over ranks; n_total (the job's primary
    count, the same on every rank) kept."""
    v = _allreduce([int(stats[k]) for k in SUMMED_STATS], np.int64, group)
    out = dict(stats)
    out.update({k: int(x) for k, x in zip(SUMMED_STATS, v)})
    return out


def run_sharded(model: "Model", n_s: float, seed: int, group=None, stream=None):
    """Runs this rank's shard of the job (N_s, seed) on its GPU and returns the job's summed
    counters and spectrum accumulators [n_incl][n_bins][3] on every rank."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    st = model.run(n_s, seed, shard=rank, n_shards=world, stream=stream)
    return allreduce_stats(st, group), allreduce_spectrum(model.spectrum_sums(), group)
