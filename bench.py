"""Benchmark of the Monte Carlo transport hot path on GB300.

Metric: superphotons tracked per second (emitted + scattered, as counted in the paper's throughput
figure, section 5).  The headline workload is the 3-D snapshot stand-in, the largest single-GPU
configuration and the shape of the paper's own throughput benchmark (section 4.3: a 288 x 128 x 128
GRMHD snapshot): a = 0.5, 288 x 128 x 128 modified Kerr-Schild grid of FP32 fields (Fishbone-Moncrief
torus x lognormal k^-11/3 turbulence), 6 inclination x 200 frequency bins, N_s = 1e8, Philox seed 1.
The headline form is plain FP64.  One step = one mc_run of one shard of that job (weights, zone
counts and scan over the whole grid, then the transport of the shard's primaries and all their
descendants, and the binning): 8 shards make one whole job, so steps 0-7 are the N_s = 1e8 job of
seed 1 (2.2e7 primaries: the weight floor w_min = 1e20 of the section 4.3 set-up keeps the count below
N_s) and later steps continue with seed 2, 3, ...  Inputs are synthetic (seeded), resident in HBM before
the timed region; L2 is flushed (256 MiB write) between timed steps.

Beside the headline the line carries, per configuration, the forms of the metric with their spectrum
error against the plain FP64 run of the same job: the 3-D snapshot in mixed precision with and without
the coefficient surrogate, the 2-D Kerr torus (256 x 128, N_s = 1e7), the scattering sphere (1024 x 128,
N_s = 1e7, four Thomson depths), the thin sphere (N_s = 1e5), and the 64-model survey batched into one
persistent launch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) the ranks share the job: at step k rank r runs shard (k N + r) mod 8, and the
ranks sum their spectrum accumulators with one allreduce per step (the path's only exchange).  Per-GPU
work is fixed: weak scaling, value = all ranks' superphotons / slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "superphotons tracked/sec on 1 GB300: plain FP64 vs batched+surrogate at <=1% spectrum err"
UNIT = "superphotons/s"
N_S_C4 = 1e8
SHARDS = 8
WORKLOAD_C4 = ("synthetic 3-D snapshot: Kerr a=0.5, modified Kerr-Schild 288x128x128 (r from horizon to 40, "
               "hslope 0.3), FP32 fields: Fishbone-Moncrief torus x lognormal k^-11/3 turbulence (sigma 0.1), "
               "R_high=20, M_unit=1e18 g, w_min=1e20, bias 96e4 Theta_e^2 (<= 1e5), N_s=1e8 per job (8 shards), "
               "200 log bins 1e8-1e24 Hz x 6 inclination bins")
WORKLOAD_C3 = "synthetic 2-D torus: Kerr a=0.9375, MKS 256x128, FP64 fields, R_high=20, N_s=1e7, seed 1"
WORKLOAD_C2 = ("scattering synchrotron sphere, Schwarzschild a=0, R=10 GM/c^2, Theta_e=4, B=10 G, "
               "tau_T in {1e-4,1e-3,1e-2,1e-1}, grid 1024x128, N_s=1e7 per run, seed 1")
WORKLOAD_C1 = "thin synchrotron sphere, Schwarzschild a=0, R=10 GM/c^2, Theta_e=10, B=10 G, grid 1024x128, N_s=1e5, seed 1"
SURVEY = ("batched parameter survey: 64 synthetic 2-D Fishbone-Moncrief tori drawn (seed 1) from spin "
          "{-0.94,-0.5,0,0.5,0.94} x R_high {1,10,40,160} x accretion scale {0.5,1,2,4} (M_unit = 5e17 g x scale), "
          "grids 128x64 / 192x96 / 256x128, N_s log-uniform in [1e5, 1e7] per model, bias 96e4 Theta_e^2 (<= 1e5)")

# ---------------------------------------------------------------------------------------------
# Algorithmic operation counts (add/mul/div/sqrt = 1, FMA = 2, each transcendental = 1), itemised
# from the formulas each kernel form evaluates.  The spin form is the one the library launches: the
# Schwarzschild form (a = 0) leaves out the terms that vanish at a = 0; 3-D grids blend 8 corners.
OPS_STEPSIZE = 10          # 1 / (|k1|/d1 + |k2|/d2 + |k3|/d3) in one division
OPS_POSITION = 28          # x_{n+1} = x_n + k dl + dl^2/2 a (4 components) and the predictor start
OPS_METRIC = {"kerr": 135, "schw": 59}      # metric, inverse and x1/x2 derivatives at x_{n+1}
OPS_INTERP = {2: 80, 3: 150}                 # 8 primitives blended over 4 (2-D) or 8 (3-D) corners
OPS_PLASMA = {"kerr": 90, "schw": 80}       # u^mu from U^i, b^mu, b^2, n_e, |B|, Theta_e
OPS_COEFF = 80             # nu_f, cos theta_B, j_nu (fit), B_nu, alpha_nu, K2 and sigma_h lookups
OPS_DEPTH = 20             # trapezoid optical depths, weight update, biased scattering depth
OPS_TERM = 5               # record / capture / roulette tests
OPS_ACCEL = {"kerr": 74, "schw": 39}        # dk/dl = -Gamma k k from the contracted derivatives
OPS_VERLET = 24            # k_{n+1} = k_n + dl/2 (a_n + a_{n+1}) and the L1 convergence test
OPS_EVENT = 30             # scattering event located by linear fraction, child written (in-grid kernel)
OPS_CHILD_LOAD = 1500      # Compton kinematics at child load (tetrad, electron, Klein-Nishina, boosts)
OPS_EMIT = 2000            # emission: frequency and direction rejection, tetrad, k^mu


def ops_grid_step(spin, dim):
    """FP64 in-grid step outside the predictor loop."""
    return (OPS_STEPSIZE + OPS_POSITION + OPS_METRIC[spin] + OPS_INTERP[dim] + OPS_PLASMA[spin] + OPS_COEFF
            + OPS_DEPTH + OPS_TERM)


def ops_geodesic_step(spin):
    """Geodesic part of a step (the whole free-streaming step; the FP64-level part of a mixed step)."""
    return OPS_STEPSIZE + OPS_POSITION + OPS_METRIC[spin] + OPS_TERM


def ops_pass(spin):
    return OPS_ACCEL[spin] + OPS_VERLET


GEN_LAUNCHES = 7          # zone prep, weight partials, weight final, counts, 3 scan kernels
FLOP_SUR_EVAL = 2.0 * (3 * 64 + 64 * 64 + 64 * 3)   # one 3-64-64-3 network evaluation (algorithmic)
# The mixed-precision forms run the geodesic in double-float on the FP32 pipes.  FP32 flops per
# FP64-equivalent operation of the hand count, from the library's double-float arithmetic (FMA = 2):
# a term of a one-pass sum of products (a product and an addition, 2 operations) is 15 (a product,
# three FMAs, a two-sum, two additions), 7.5 per operation; a separate Dekker sum is 11 and a separate
# product 10.  The geodesic's accelerations, Verlet updates and metric body are sums of products, the
# rest separate sums and products: about 9 per operation (an estimate; the ncu pipe figures below are
# the measured counterpart).
DF_FLOPS_PER_OP = 9.0

# DRAM bytes (read + write) per superphoton handed to the in-grid kernel, from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch / superphotons it carried); traffic grows
# in proportion to the superphotons a launch carries.  Keyed by (workload, form); re-taken whenever
# the kernel changes (profiles/ holds the summaries).
TRAFFIC_B_PER_PH = {("c4", "fp64"): 6641.8}
# ncu-measured pipe utilisation of the double-float in-grid kernel (a full capture of its first launch
# on the 3-D snapshot at N_s = 4e6): FP32 and FP64 pipes busy, issue active.
NCU_MIXED_FP32_PIPE = {"in_grid_fp32": 0.257, "in_grid_fp64": 0.159, "issue_active": 0.370,
                       "source": "ncu, 3-D snapshot N_s=4e6, k_push_mixed<0,1> at 8 CTAs/SM, FP32 weights"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), d.get("bf16_tflops"), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, 1900.0, "fallback"


# ---------------------------------------------------------------------------------------------
def oracle_sample(om, tot, uid0, uid1, budget_s, nthreads, n0=256):
    """Times the CPU oracle as it stands on a bounded sample: the first primaries of [uid0, uid1) of a
    prepared job and all their descendants, grown until the sample takes ~budget_s."""
    n = n0
    while True:
        t = time.perf_counter()
        r = om.run(uid0, min(uid0 + n, uid1), nthreads=nthreads)
        dt = time.perf_counter() - t
        if dt > 0.3 * budget_s or uid0 + n >= uid1:
            break
        n = int(n * min(8.0, max(2.0, 0.5 * budget_s / max(dt, 1e-3))))
    st = r["stats"]
    units = st["n_emit"] + st["n_child"]
    return units / dt, units, dt, min(n, uid1 - uid0)


def shard_range(tot, shard, n_shards):
    return (tot * shard) // n_shards, (tot * (shard + 1)) // n_shards


def spectrum_error(s_new, s_ref, min_count=16):
    """Error of one spectrum against the plain FP64 spectrum of the same job: relative error of the
    total luminosity, the number of bins compared (>= min_count superphotons on both sides), and how
    many of them are within max(1 %, 3 combined Monte Carlo sigma)."""
    import numpy as np
    a, b = s_new[..., 0], s_ref[..., 0]
    tot = float(b.sum())
    lum = abs(float(a.sum()) - tot) / tot if tot > 0 else 0.0
    sig = np.sqrt(s_new[..., 1] + s_ref[..., 1])
    sel = (s_new[..., 2] >= min_count) & (s_ref[..., 2] >= min_count)
    ok = np.abs(a - b) <= np.maximum(0.01 * np.abs(b), 3.0 * sig)
    return lum, int(sel.sum()), int((sel & ok).sum())


def error_block(pairs):
    import numpy as np
    errs = [spectrum_error(a, b) for a, b in pairs]
    lum = [e[0] for e in errs]
    nb, nok = sum(e[1] for e in errs), sum(e[2] for e in errs)
    return {"total_luminosity_rel_max": max(lum), "total_luminosity_rel_median": float(np.median(lum)),
            "bins_within_max_1pct_3sigma": nok / max(nb, 1), "bins_compared": nb, "within_1pct": bool(max(lum) <= 0.01)}


def sum_stats(stats):
    out = {}
    for s in stats:
        for k, v in s.items():
            if isinstance(v, (int, float)):
                out[k] = out.get(k, 0) + v
    return out


def fp64_roofline(st, spin, dim, fp64_peak, kernel, traffic_per_ph=None, hbm_peak=None, fp32_peak=None):
    """In-grid FP64 kernel against the measured FP64 FMA peak: achieved = the itemised count of the
    form that ran x the step, pass and event counters / the in-grid phase's event-timed duration."""
    t_grid = st["grid_ms"] / 1e3
    ops = (ops_grid_step(spin, dim) * st["n_steps_grid"] + ops_pass(spin) * st["n_iters_grid"]
           + OPS_EVENT * st["n_events"])
    ach = ops / t_grid
    r = {"bound": "alu", "achieved": ach / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": ach / fp64_peak,
         "traffic": None, "kernel": kernel,
         "count": {"spin_form": spin, "grid_dim": dim, "ops_per_in_grid_step": ops_grid_step(spin, dim),
                   "ops_per_predictor_pass": ops_pass(spin), "ops_per_event": OPS_EVENT,
                   "in_grid_steps": st["n_steps_grid"], "predictor_passes": st["n_iters_grid"], "events": st["n_events"]},
         "peak_source": "measured: project FP64 FMA-chain microbenchmark on this GPU (mc_fma_peak)",
         "phase_s": {"init": st["init_ms"] / 1e3, "in_grid": t_grid, "free": st["free_ms"] / 1e3}}
    if fp32_peak:
        r["fp32_peak_tflops"] = fp32_peak / 1e12
    if traffic_per_ph and hbm_peak:
        # traffic of the first in-grid launch of each run: it carries every primary of the run
        tb = traffic_per_ph * st["n_emit"]
        r["traffic"] = tb
        r["traffic_note"] = ("ncu DRAM read+write per superphoton (%.1f B) x primaries handed to the first in-grid "
                             "launch of each run" % traffic_per_ph)
        r["hbm"] = {"achieved_gbs": tb / t_grid / 1e9, "peak_gbs": hbm_peak, "frac": tb / t_grid / 1e9 / hbm_peak}
    return r


def split_roofline(st, spin, fp64_peak, kernel, phase="in_grid"):
    """Split form (FP64 geodesic, FP32 coefficients and weights) against the measured FP64 peak: achieved =
    the FP64 geodesic operations of the in-grid phase / its duration (phase "batch": of every step over
    the whole batched transport launch); the FP32 coefficient work rides on the FP32 pipes beside it."""
    if phase == "in_grid":
        ops = ops_geodesic_step(spin) * st["n_steps_grid"] + ops_pass(spin) * st["n_iters_grid"]
        ach = ops / (st["grid_ms"] / 1e3)
    else:
        ops = ops_geodesic_step(spin) * st["n_steps"] + ops_pass(spin) * st["n_iters"]
        ach = ops / (st["transport_ms"] / 1e3)
    return {"bound": "alu", "kernel": kernel, "achieved": ach / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
            "frac": ach / fp64_peak, "traffic": None,
            "peak_source": "measured: project FP64 FMA-chain microbenchmark on this GPU (mc_fma_peak)",
            "count": {"ops_per_in_grid_step_fp64": ops_geodesic_step(spin), "ops_per_predictor_pass": ops_pass(spin),
                      "in_grid_steps": st["n_steps_grid"], "predictor_passes": st["n_iters_grid"]}}


def df_roofline(st, spin, fp32_peak, fp64_peak, kernel, phase="in_grid"):
    """Double-float kernel against the measured FP32 peak.  achieved = FP64-equivalent geodesic
    operations x DF_FLOPS_PER_OP (an estimate from the library's double-float arithmetic); the ncu-measured
    FP32-pipe busy fraction sits beside it."""
    if phase == "in_grid":
        ops = ops_geodesic_step(spin) * st["n_steps_grid"] + ops_pass(spin) * st["n_iters_grid"]
        sec = st["grid_ms"] / 1e3
    else:   # whole batched transport
        ops = (ops_geodesic_step(spin) * st["n_steps"] + ops_pass(spin) * st["n_iters"]
               + OPS_EMIT * st["n_emit"] + OPS_CHILD_LOAD * st["n_child"])
        sec = st["transport_ms"] / 1e3
    eq = ops / max(sec, 1e-30)
    fp32 = DF_FLOPS_PER_OP * eq
    return {"bound": "alu", "kernel": kernel, "achieved": fp32 / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
            "frac": fp32 / fp32_peak, "traffic": None, "peak_source": "measured FP32 FMA-chain (mc_fma_peak)",
            "note": "geodesic in double-float on the FP32 pipes; achieved = FP64-equivalent geodesic operations x "
                    "%.0f FP32 flops each (estimate)" % DF_FLOPS_PER_OP,
            "ncu_fp32_pipe_busy": NCU_MIXED_FP32_PIPE,
            "fp64_equivalent_tflops": eq / 1e12, "vs_fp64_peak": eq / fp64_peak}


# ---------------------------------------------------------------------------------------------
class Timer:
    def __init__(self, stream):
        import torch
        self.stream = stream
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)

    def run(self, fn, flush):
        import torch
        flush.zero_()
        self.e0.record(self.stream)
        r = fn()
        self.e1.record(self.stream)
        torch.cuda.synchronize()
        return r, self.e0.elapsed_time(self.e1)


def run_form(ctx, jobs, timer, flush):
    """Runs (n_s, seed, shard, n_shards) jobs on one context, each timed; returns summed counters,
    the summed spectrum accumulators per seed and the device milliseconds."""
    stats, ms, sums = [], 0.0, {}
    for n_s, seed, shard, nsh in jobs:
        st, t = timer.run(lambda: ctx.run(n_s, seed, shard=shard, n_shards=nsh, stream=timer.stream), flush)
        stats.append(st)
        ms += t
        s = ctx.spectrum_sums()
        sums[seed] = sums.get(seed, 0) + s
    return sum_stats(stats), sums, ms


def form_entry(st, ms, ref_value=None):
    u = st["n_emit"] + st["n_child"]
    r = {"value": u / (ms / 1e3), "unit": UNIT, "superphotons": int(u), "ms": ms,
         "scatterings_per_s": st["n_events"] / (ms / 1e3)}
    if ref_value:
        r["speedup_vs_plain_fp64"] = r["value"] / ref_value
    return r


def config_forms(name, p, g, jobs, spin, dim, dev, timer, flush, peaks, weights, ref=None, mixed_forms=True,
                 oracle_sums=None):
    """Plain FP64 (unless ref = (stats, sums, ms) of it is given), mixed, and mixed + surrogate forms of one
    configuration on the same jobs; spectrum errors against the plain FP64 sums of each seed, and, when
    oracle_sums (the oracle's sums of the seed-1 job) is given, against the oracle too."""
    import torch
    from paper_2602_13198_gb300 import mc
    fp64_peak, fp32_peak, hbm_peak, bf16_peak = peaks
    out = {}
    if ref is None:
        m = mc.Model(p, device=dev, precision="fp64")
        m.set_grid(g)
        m.run(min(jobs[0][0], 1e4), 999, stream=timer.stream)   # warm-up (queues, tables)
        ref = run_form(m, jobs, timer, flush)
        del m
    st0, sums0, ms0 = ref
    e = form_entry(st0, ms0)
    e["roofline"] = fp64_roofline(st0, spin, dim, fp64_peak, "k_push_fp64<in-grid, %s>" % spin,
                                  TRAFFIC_B_PER_PH.get((name, "fp64")), hbm_peak)
    if oracle_sums is not None and 1 in sums0:
        e["spectrum_error_vs_oracle"] = error_block([(sums0[1], oracle_sums)])
    out["plain_fp64"] = e
    if not mixed_forms:
        return out
    for form, prec, sur in (("mixed", "mixed", False), ("mixed_surrogate", "mixed", True), ("split", "split", False),
                            ("split_surrogate", "split", True)):
        if sur and (weights is None or p.get("kappa", 0) or p.get("brems", 0)):
            continue
        m = mc.Model(p, device=dev, precision=prec, surrogate=sur)
        if sur:
            m.surrogate_weights(weights)
        m.set_grid(g)
        m.run(min(jobs[0][0], 1e4), 999, stream=timer.stream)
        st, sums, ms = run_form(m, jobs, timer, flush)
        del m
        torch.cuda.empty_cache()
        e = form_entry(st, ms, out["plain_fp64"]["value"])
        e["spectrum_error"] = error_block([(sums[s], sums0[s]) for s in sums])
        if oracle_sums is not None and 1 in sums:
            e["spectrum_error_vs_oracle"] = error_block([(sums[1], oracle_sums)])
        if prec == "split":
            e["roofline"] = split_roofline(st, spin, fp64_peak, "k_push_%s<in-grid, %s> (FP64 geodesic, FP32 rest)"
                                           % ("sur" if sur else "split", spin))
        else:
            e["roofline"] = df_roofline(st, spin, fp32_peak, fp64_peak,
                                        "k_push_%s<in-grid, %s> (double-float geodesic)" % ("sur" if sur else "mixed", spin))
        if sur:
            tf = FLOP_SUR_EVAL * st["n_steps_grid"] / (st["grid_ms"] / 1e3) / 1e12
            e["surrogate"] = {"tensor_achieved_tflops": tf, "bf16_peak_tflops": bf16_peak,
                              "tensor_frac": tf / bf16_peak if bf16_peak else None, "evals": st["n_steps_grid"]}
        out[form] = e
    return out


def survey_forms(args, dev, timer, flush, peaks, weights):
    """The metric's second form on the survey workload: the same 64 models and seeds run (1) as plain
    FP64, one mc_run per model, and (2) batched into one persistent launch (autotuned, replayed from
    a captured CUDA graph) in mixed precision, with and without the coefficient surrogate."""
    import torch
    from paper_2602_13198_gb300 import mc, synth
    fp64_peak, fp32_peak, hbm_peak, bf16_peak = peaks
    specs = synth.survey(64, 1)
    ns = [n * args.survey_scale for (_, _, n) in specs]
    seeds = [1 + i for i in range(len(specs))]
    out = {"workload": SURVEY, "n_s_scale": args.survey_scale, "n_s_total": sum(ns), "models": len(specs)}
    ref, stats, ms, launches = [], [], 0.0, 0
    for (p, g, _), n_s, sd in zip(specs, ns, seeds):
        m = mc.Model(p, device=dev, precision="fp64")
        m.set_grid(g)
        m.run(min(n_s, 1e4), sd, stream=timer.stream)
        st, t = timer.run(lambda: m.run(n_s, sd, stream=timer.stream), flush)
        stats.append(st)
        ms += t
        launches += st["transport_launches"] + GEN_LAUNCHES
        ref.append(m.spectrum_sums().copy())
        del m
    torch.cuda.empty_cache()
    st0 = sum_stats(stats)
    out["emitting_models"] = sum(1 for s in stats if s["n_total"] > 0)
    out["plain_fp64"] = dict(form_entry(st0, ms), gpu_launches=launches)
    for form, prec, sur in (("batched_mixed", "mixed", False), ("batched_mixed_surrogate", "mixed", True),
                            ("batched_split_surrogate", "split", True)):
        ctxs = []
        for (p, g, _) in specs:
            m = mc.Model(p, device=dev, precision=prec, surrogate=sur)
            if sur:
                m.surrogate_weights(weights)
            m.set_grid(g)
            ctxs.append(m)
        t0 = time.perf_counter()
        mc.run_batch(ctxs, ns, seeds, autotune=True, graph=True, stream=timer.stream)   # tune + capture
        t_setup = time.perf_counter() - t0
        st, bms = timer.run(lambda: mc.run_batch(ctxs, ns, seeds, autotune=True, graph=True, stream=timer.stream), flush)
        r = form_entry(st, bms, out["plain_fp64"]["value"])
        r["spectrum_error"] = error_block([(c.spectrum_sums(), rr) for c, rr in zip(ctxs, ref)])
        r["autotune"] = {"min_blocks_per_sm": st["batch_min_blocks"], "ctas": st["batch_ctas"],
                         "graph": bool(st["batch_graph"]), "tune_and_capture_s": t_setup}
        r["gpu_launches"] = 1 + GEN_LAUNCHES * len(specs) + 1
        if prec == "split":
            r["roofline"] = split_roofline(st, "kerr", fp64_peak, "k_batch (whole batched transport, one cooperative "
                                           "launch, FP64 geodesic; Kerr count for every model)", phase="batch")
        else:
            r["roofline"] = df_roofline(st, "kerr", fp32_peak, fp64_peak, "k_batch (whole batched transport, one "
                                        "cooperative launch; Kerr count for every model)", phase="batch")
        if sur:
            tf = FLOP_SUR_EVAL * st["n_steps_grid"] / (st["transport_ms"] / 1e3) / 1e12
            r["surrogate"] = {"tensor_achieved_tflops": tf, "bf16_peak_tflops": bf16_peak,
                              "tensor_frac": tf / bf16_peak if bf16_peak else None, "evals": st["n_steps_grid"]}
        out[form] = r
        del ctxs
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------------------------
def grid_dims(args):
    n1, n2, n3 = (int(x) for x in args.grid.split("x"))
    return {} if (n1, n2, n3) == (288, 128, 128) else {"n1": n1, "n2": n2, "n3": n3}


def reference_arm(args, cores):
    """The reference arm is the CPU oracle (no reference implementation exists to install): the main
    workload's job prepared once (weights and counts over the whole grid), then per step a bounded
    sample of the step's shard (its first primaries and their descendants) on all host cores."""
    import numpy as np

    import oracle
    from paper_2602_13198_gb300 import synth
    oracle.build()
    p, g = synth.torus3d(**grid_dims(args))
    go = dict(g, prim=np.asarray(g["prim"], dtype=np.float64))
    om = oracle.Model(p, go)
    t0 = time.perf_counter()
    tot = om.prepare(args.n_s, 1)
    t_prep = time.perf_counter() - t0
    for w in range(args.warmup):
        u0, u1 = shard_range(tot, w % args.shards, args.shards)
        om.run(u0, min(u1, u0 + 16), nthreads=cores)
    units, secs, samples = 0, 0.0, []
    for k in range(args.steps):
        u0, u1 = shard_range(tot, k % args.shards, args.shards)
        rate, u, dt, n = oracle_sample(om, tot, u0, u1, 4.0, cores)
        units += u
        secs += dt
        samples.append(n)
    v = units / secs
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_C4 if not grid_dims(args) else WORKLOAD_C4 + " (grid " + args.grid + ")",
                       "form": "plain FP64 (CPU oracle)", "n_s_per_job": args.n_s,
                       "shards_per_job": args.shards},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step the first %s primaries (and their scattered descendants) of that step's "
                                       "shard of the seed-1 job; weights and counts of the 4.7M-zone grid prepared once "
                                       "beforehand (%.0f s, not in the rate)" % (samples, t_prep)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-s", type=float, default=N_S_C4, help="N_s of the main job (smaller for profiling)")
    ap.add_argument("--shards", type=int, default=SHARDS, help="shards per job (one per step)")
    ap.add_argument("--grid", default="288x128x128", help="3-D grid of the main workload (smaller for tests)")
    ap.add_argument("--main-precision", default="fp64", choices=["fp64", "mixed", "split"],
                    help="precision form of the main line (profiling; the headline is plain FP64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass (profiling runs)")
    ap.add_argument("--no-forms", action="store_true", help="skip the per-configuration forms")
    ap.add_argument("--no-survey", action="store_true", help="skip the batched-survey form")
    ap.add_argument("--survey-scale", type=float, default=1.0, help="N_s multiplier of the survey form")
    ap.add_argument("--forms-scale", type=float, default=1.0, help="N_s multiplier of the 2-D configuration forms")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cores = os.cpu_count() or 1
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(args, cores)), flush=True)
        return

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2602_13198_gb300 import build, mc, synth
    build.build()
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    fp64_peak = mc.fma_peak(dev, True)
    fp32_peak = mc.fma_peak(dev, False)
    hbm_peak, bf16_peak, peak_src = measured_peaks()
    peaks = (fp64_peak, fp32_peak, hbm_peak, bf16_peak)
    timer = Timer(stream)

    # ---- main workload: the 3-D snapshot, plain FP64, one shard of the job per step
    p4, g4 = synth.torus3d(**grid_dims(args))
    m4 = mc.Model(p4, device=dev, precision=args.main_precision)
    m4.set_grid(g4)
    S = args.shards

    def job_of(k):
        j = k * world + rank
        return 1 + j // S, j % S

    def one(k):
        seed, shard = job_of(k)
        st = m4.run(args.n_s, seed, shard=shard, n_shards=S, stream=stream)
        if dist:
            sums = torch.from_numpy(m4.spectrum_sums()).cuda()
            dist.all_reduce(sums)
        return st

    for w in range(args.warmup):
        one(w)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(dev)
    sampler.start()
    stats, step_ms, sums_by_seed = [], [], {}
    t_wall = time.perf_counter()
    for k in range(args.steps):
        st, t = timer.run(lambda: one(k), flush)
        stats.append(st)
        step_ms.append(t)
        seed, _ = job_of(k)
        sums_by_seed[seed] = sums_by_seed.get(seed, 0) + m4.spectrum_sums()   # outside the timed events
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    dev_s = sum(step_ms) / 1e3
    st_main = sum_stats(stats)
    units = st_main["n_emit"] + st_main["n_child"]
    launches = st_main["transport_launches"] + GEN_LAUNCHES * args.steps
    if dist:
        t = torch.tensor([dev_s, float(units)], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        dev_s_max, units_all = float(tmax[0]), float(t[1])
    else:
        dev_s_max, units_all = dev_s, float(units)
    value = units_all / dev_s_max

    # ---- end to end through the public API with host buffers: grid H2D each step, spectrum D2H
    host_prim = torch.from_numpy(np.ascontiguousarray(g4["prim"])).pin_memory()
    e2e_units, t_e2e = 0, 1e-300
    for k in range(0 if args.no_e2e else args.steps):
        seed, shard = job_of(k)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m4.set_grid(g4, prim=host_prim.numpy())
        s = m4.run(args.n_s, seed, shard=shard, n_shards=S, stream=stream)
        m4.spectrum()
        t_e2e += time.perf_counter() - t0
        e2e_units += s["n_emit"] + s["n_child"]
    h2d = int(host_prim.numel() * host_prim.element_size())
    d2h = int(m4.n_incl * m4.n_bins * 3 * 8)
    if dist:
        t = torch.tensor([t_e2e, float(e2e_units)], dtype=torch.float64, device="cuda")
        tm = t.clone()
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        e2e_value = float(t[1]) / float(tm[0])
    else:
        e2e_value = e2e_units / t_e2e

    share = 100 * st_main["grid_ms"] / max(st_main["transport_ms"], 1e-30)
    if args.main_precision == "mixed":
        roofline = df_roofline(st_main, "kerr", fp32_peak, fp64_peak, "k_push_mixed<in-grid, kerr>: %.0f%% of transport "
                               "time" % share)
    elif args.main_precision == "split":
        roofline = split_roofline(st_main, "kerr", fp64_peak, "k_push_split<in-grid, kerr>: %.0f%% of transport time"
                                  % share)
    else:
        roofline = fp64_roofline(st_main, "kerr", 3, fp64_peak, "k_push_fp64<in-grid, kerr> (FP64, trilinear FP32 "
                                 "fields): dominant kernel, %.0f%% of transport time" % share,
                                 TRAFFIC_B_PER_PH.get(("c4", "fp64")), hbm_peak, fp32_peak)

    cpu = None
    oracle_c1_spec = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        go = dict(g4, prim=np.asarray(g4["prim"], dtype=np.float64))
        om = oracle.Model(p4, go)
        t0 = time.perf_counter()
        tot = om.prepare(args.n_s, 1)
        t_prep = time.perf_counter() - t0
        u0, u1 = shard_range(tot, 0, S)
        rate, u, dt, n = oracle_sample(om, tot, u0, u1, 12.0, cores)
        rate1, u_1, dt1, n1 = oracle_sample(om, tot, u0, u1, 8.0, 1, n0=16)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "first %d primaries (+ scattered descendants: %d superphotons) of shard 0 of the seed-1 job, "
                         "%.1f s on %d threads; weights and counts of the grid prepared once (%.0f s, not in the rate)"
                         % (n, u, dt, cores, t_prep),
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": "first %d primaries (%d superphotons) of the same shard, %.1f s"
                                           % (n1, u_1, dt1)}}
        del om
        # the oracle on the other configurations' workloads (bounded samples, all cores), beside the
        # device forms of the same jobs
        per = {}
        for cname, (pc, gc), n_s in (("c3_torus_2d", synth.torus(), 1e7),
                                     ("c2_scattering_sphere_tau_0.1", synth.scattering_sphere(1e-1), 1e7)):
            omc = oracle.Model(pc, gc)
            totc = omc.prepare(n_s, 1)
            rc, uc, dtc, nc = oracle_sample(omc, totc, 0, totc, 3.0, cores)
            per[cname] = {"value": rc, "unit": UNIT, "cores": cores,
                          "sample": "first %d primaries (%d superphotons) of the seed-1 job at N_s = %.0e, %.1f s"
                                    % (nc, uc, n_s, dtc)}
            del omc
        # the thin sphere's whole job (N_s = 1e5): its spectrum is also the oracle reference of the
        # thin-sphere forms below
        omc = oracle.Model(*synth.sphere("ks"))
        omc.prepare(1e5, 1)
        t0 = time.perf_counter()
        rc1 = omc.run(nthreads=cores)
        dtc = time.perf_counter() - t0
        uc = rc1["stats"]["n_emit"] + rc1["stats"]["n_child"]
        oracle_c1_spec = rc1["spec"]
        per["c1_thin_sphere"] = {"value": uc / dtc, "unit": UNIT, "cores": cores,
                                 "sample": "the whole seed-1 job at N_s = 1e5 (%d superphotons), %.1f s" % (uc, dtc)}
        del omc
        cpu["per_config"] = per

    forms = None
    if world == 1 and not args.no_forms and args.main_precision == "fp64":
        forms = {"peaks": {"fp64_tflops": fp64_peak / 1e12, "fp32_tflops": fp32_peak / 1e12,
                           "hbm_gbs": hbm_peak, "bf16_tflops": bf16_peak, "hbm_bf16_source": peak_src}}
        # the coefficient network, trained on the GPU by the library's own kernels (untimed set-up)
        trainer = mc.Model(synth.sphere("flat", n1=4, n2=4)[0], device=dev, precision="mixed")
        t0 = time.perf_counter()
        vloss = trainer.surrogate_train(n_train=1 << 18, steps=40000, batch=4096, lr=2e-3, seed=1)
        weights = trainer.surrogate_weights()
        forms["surrogate_training"] = {"validation_loss": vloss, "s": time.perf_counter() - t0}
        del trainer
        # 3-D snapshot: the FP64 reference is the whole job of seed 1 (the timed shards, completed here)
        done = [job_of(k) for k in range(args.steps)]
        for sh in range(S):
            if (1, sh) not in done:
                m4.run(args.n_s, 1, shard=sh, n_shards=S, stream=stream)
                sums_by_seed[1] = sums_by_seed.get(1, 0) + m4.spectrum_sums()
        st_ref = sum_stats([s for s, k in zip(stats, range(args.steps)) if job_of(k)[0] == 1])
        ms_ref = sum(t for t, k in zip(step_ms, range(args.steps)) if job_of(k)[0] == 1)
        jobs4 = [(args.n_s, 1, sh, S) for sh in range(S)]
        if all((1, sh) in done for sh in range(S)):
            ref4 = (st_ref, {1: sums_by_seed[1]}, ms_ref)
            forms["c4_snapshot_3d"] = config_forms("c4", p4, g4, jobs4, "kerr", 3, dev, timer, flush, peaks, weights,
                                                   ref=ref4)
        else:   # fewer timed steps than one job: time the FP64 job here
            forms["c4_snapshot_3d"] = config_forms("c4", p4, g4, jobs4, "kerr", 3, dev, timer, flush, peaks, weights)
        forms["c4_snapshot_3d"]["workload"] = WORKLOAD_C4
        del m4
        torch.cuda.empty_cache()
        fs = args.forms_scale
        p3, g3 = synth.torus()
        forms["c3_torus_2d"] = dict(config_forms("c3", p3, g3, [(1e7 * fs, 1, 0, 1)], "kerr", 2, dev, timer, flush,
                                                 peaks, weights), workload=WORKLOAD_C3)
        jobs2 = []
        c2 = {}
        for tau in (1e-4, 1e-3, 1e-2, 1e-1):
            c2[tau] = synth.scattering_sphere(tau)
        res2 = {}
        for tau, (p, g) in c2.items():
            res2[tau] = config_forms("c2", p, g, [(1e7 * fs, 1, 0, 1)], "schw", 2, dev, timer, flush, peaks, weights)
        agg = {}
        for form in res2[1e-1]:
            vals = [res2[t][form] for t in res2 if form in res2[t]]
            u = sum(v["superphotons"] for v in vals)
            ms = sum(v["ms"] for v in vals)
            agg[form] = {"value": u / (ms / 1e3), "unit": UNIT, "superphotons": u, "ms": ms,
                         "per_tau": {str(t): res2[t][form] for t in res2 if form in res2[t]}}
            if form != "plain_fp64":
                agg[form]["speedup_vs_plain_fp64"] = agg[form]["value"] / agg["plain_fp64"]["value"]
        forms["c2_scattering_sphere"] = dict(agg, workload=WORKLOAD_C2)
        p1, g1 = synth.sphere("ks")
        forms["c1_thin_sphere"] = dict(config_forms("c1", p1, g1, [(1e5, 1, 0, 1)], "schw", 2, dev, timer, flush,
                                                    peaks, weights, oracle_sums=oracle_c1_spec), workload=WORKLOAD_C1)
        if not args.no_survey:
            forms["c5_survey"] = survey_forms(args, dev, timer, flush, peaks, weights)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * dev_s_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "mixed": "f32 pairs (double-float) + f32", "split": "f64 + f32"}[args.main_precision],
                "data": "synthetic",
                "config": {"workload": WORKLOAD_C4 if not grid_dims(args) else WORKLOAD_C4 + " (grid " + args.grid + ")",
                           "form": {"fp64": "plain FP64", "mixed": "mixed (double-float geodesic)",
                                    "split": "split (FP64 geodesic, FP32 rest)"}[args.main_precision],
                           "n_s_per_job": args.n_s,
                           "shards_per_job": S, "step": "one mc_run of one shard (generation over the whole grid + "
                                                        "the shard's transport and binning)",
                           "grid": [int(x) for x in args.grid.split("x")],
                           "l2": "flushed (256 MiB write) between timed steps",
                           "parallelism": ("sharded job: rank r runs shard (k N + r) mod %d at step k, spectrum "
                                           "allreduce per step" % S) if world > 1 else "single GPU"},
                "clocks": clocks,
                "e2e": None if args.no_e2e else {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                                                  "d2h_bytes_per_step": d2h},
                "roofline": roofline, "cpu_baseline": cpu, "forms": forms,
                "gpu_launches": int(launches),
                "detail": {"superphotons": units, "scattered": st_main["n_child"],
                           "steps_per_superphoton": st_main["n_steps"] / max(units, 1),
                           "iters_per_step": st_main["n_iters"] / max(1, st_main["n_steps"]),
                           "step_ms": step_ms, "wall_s": t_wall,
                           "generate_ms": [s["generate_ms"] for s in stats],
                           "scatterings_per_s": st_main["n_events"] / dev_s}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
