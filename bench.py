"""Benchmark of the Monte Carlo transport hot path on GB300.

Metric: superphotons tracked per second (emitted + scattered, as counted in the paper's
throughput figure), plain FP64 form, on the scattering synchrotron sphere: Schwarzschild
sphere of radius 10 GM/c^2, Theta_e = 4, B = 10 G, 1024 x 128 grid, Thomson depth
tau_T in {1e-4, 1e-3, 1e-2, 1e-1}, N_s = 1e7 per run, seeds 1-4.  One step = one whole
mc_run (weights, zone counts, emission, transport of every generation, binning) of one
(tau_T, seed) pair, cycling through the 16 pairs.  Inputs are synthetic (seeded), resident in
HBM before the timed region; L2 is flushed (256 MiB write) between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) each rank runs its own independent jobs (seed offset by rank; no
collective on the data path): weak scaling, value = all ranks' superphotons / slowest rank time.
"""
from __future__ import annotations

import argparse
import json
import math
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
TAUS = (1e-4, 1e-3, 1e-2, 1e-1)
N_S = 1e7
WORKLOAD = ("scattering synchrotron sphere, Schwarzschild a=0, R=10 GM/c^2, Theta_e=4, B=10 G, "
            "tau_T in {1e-4,1e-3,1e-2,1e-1}, grid 1024x128, N_s=1e7 per run, seeds 1-4, 200 log bins 1e8-1e24 Hz")

# Algorithmic FP64 operations (add/mul/div/sqrt = 1, FMA = 2, each transcendental = 1), hand-counted
# from the formulas of the FP64 path.  In-grid step outside the predictor loop: step size (8),
# position update (28), metric and its x1/x2 derivatives (130), fluid interpolation (80), plasma
# state (90), j_nu / B_nu / sigma_h (80), optical depths and weight update (20), termination (5);
# free-streaming step: step size, position update, metric derivatives, termination (170); each
# Verlet predictor pass (acceleration contraction + convergence test): 110; emission: 2000;
# scattering event (kinematics + tetrad + child): 1500.  Mixed form: the in-grid coefficients run in
# FP32, leaving 190 FP64 operations per in-grid step.
FLOP_STEP_GRID = 460.0
FLOP_STEP_GRID_MIXED = 190.0
FLOP_STEP_FREE = 170.0
FLOP_ITER = 110.0
FLOP_EMIT = 2000.0
FLOP_EVENT = 1500.0
GEN_LAUNCHES = 7          # zone prep, weight partials, weight final, counts, 3 scan kernels
# DRAM bytes (read + write) per superphoton of the first in-grid launch of a job, from one ncu capture
# of k_push_fp64<in-grid> at N_s = 1e6, tau_T = 1e-2 (224.9 MB for ~787k superphotons); traffic grows
# in proportion to the superphotons a launch carries.  Must be re-taken whenever that kernel changes.
TRAFFIC_B_PER_PH_FP64 = 285.9


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


def oracle_rate(p, g, seed, budget_s, nthreads, first_n=None):
    """Times the CPU oracle as it stands on a bounded sample (the first uids of the job)."""
    import oracle
    om = oracle.Model(p, g)
    tot = om.prepare(N_S, seed)
    n = first_n or 256
    while True:
        t = time.perf_counter()
        r = om.run(0, min(n, tot), nthreads=nthreads)
        dt = time.perf_counter() - t
        if first_n or dt > 0.3 * budget_s or n >= tot:
            break
        n = int(n * min(8.0, max(2.0, 0.5 * budget_s / max(dt, 1e-3))))
    st = r["stats"]
    units = st["n_emit"] + st["n_child"]
    return units / dt, units, dt, min(n, tot)


SURVEY = ("batched parameter survey: 64 synthetic 2-D Fishbone-Moncrief tori drawn (seed 1) from spin "
          "{-0.94,-0.5,0,0.5,0.94} x R_high {1,10,40,160} x accretion scale {0.5,1,2,4} (M_unit = 5e17 g x scale), "
          "grids 128x64 / 192x96 / 256x128, N_s log-uniform in [1e5, 1e7] per model, bias 96e4 Theta_e^2 (<= 1e5)")
FLOP_SUR_EVAL = 2.0 * (3 * 64 + 64 * 64 + 64 * 3)   # one 3-64-64-3 network evaluation (algorithmic)
# The mixed-precision forms run the geodesic in double-float on the FP32 pipes.  FP32 flops per
# FP64-equivalent operation of the hand count, from the library's double-float arithmetic: an
# addition is 20 (two two-sums, two fast two-sums, two additions), a product 10 (a product, three
# FMAs at 2, a fast two-sum); the geodesic's mix of the two averages about 15.
DF_FLOPS_PER_OP = 15.0


def df_roofline(ops, seconds, fp32_peak, fp64_peak, kernel):
    """Roofline of a double-float transport kernel against the measured FP32 peak (estimate: the hand
    count's FP64-equivalent operations x DF_FLOPS_PER_OP), with the FP64-accurate operation rate beside
    it and its ratio to what the FP64 pipe could sustain."""
    eq = ops / seconds
    fp32 = DF_FLOPS_PER_OP * eq
    return {"bound": "alu", "kernel": kernel, "achieved": fp32 / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
            "frac": fp32 / fp32_peak, "peak_source": "measured FP32 FMA-chain (mc_fma_peak)",
            "note": "geodesic in double-float on the FP32 pipes; achieved = hand-counted FP64-equivalent "
                    "operations x %.0f FP32 flops each (estimate)" % DF_FLOPS_PER_OP,
            "fp64_equivalent_tflops": eq / 1e12, "vs_fp64_peak": eq / fp64_peak}


def spectrum_error(s_new, s_ref, min_count=16):
    """Error of one spectrum against the plain FP64 spectrum of the same model and seed: relative
    error of the total luminosity, and the fraction of bins (>= min_count superphotons on both
    sides) within max(1 %, 3 combined Monte Carlo sigma)."""
    import numpy as np
    a, b = s_new[..., 0], s_ref[..., 0]
    tot = float(b.sum())
    lum = abs(float(a.sum()) - tot) / tot if tot > 0 else 0.0
    sig = np.sqrt(s_new[..., 1] + s_ref[..., 1])
    sel = (s_new[..., 2] >= min_count) & (s_ref[..., 2] >= min_count)
    ok = np.abs(a - b) <= np.maximum(0.01 * np.abs(b), 3.0 * sig)
    return lum, int(sel.sum()), int((sel & ok).sum())


def survey_forms(args, dev, stream, flush, fp64_peak, fp32_peak, bf16_peak):
    """The metric's second form on the survey workload: the same 64 models and seeds run (1) as plain
    FP64, one mc_run per model, and (2) batched into one persistent launch (autotuned, replayed from
    a captured CUDA graph) in mixed precision, with and without the coefficient surrogate.  Each
    timed pass is preceded by an L2 flush and timed with CUDA events on the launching stream."""
    import numpy as np
    import torch
    from paper_2602_13198_gb300 import mc, synth
    specs = synth.survey(64, 1)
    ns = [n * args.survey_scale for (_, _, n) in specs]
    seeds = [1 + i for i in range(len(specs))]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": SURVEY, "n_s_scale": args.survey_scale, "n_s_total": sum(ns), "models": len(specs)}

    # (1) plain FP64, one model after another
    ref, units, ms, launches, events = [], 0, 0.0, 0, 0
    for (p, g, _), n_s, sd in zip(specs, ns, seeds):
        m = mc.Model(p, device=dev, precision="fp64")
        m.set_grid(g)
        m.run(min(n_s, 1e4), sd, stream=stream)       # warm-up (queues, tables)
        flush.zero_()
        e0.record(stream)
        st = m.run(n_s, sd, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        units += st["n_emit"] + st["n_child"]
        events += st["n_events"]
        launches += st["transport_launches"] + GEN_LAUNCHES
        ref.append(m.spectrum_sums().copy())
        del m
    torch.cuda.empty_cache()
    out["plain_fp64"] = {"value": units / (ms / 1e3), "unit": UNIT, "superphotons": units, "ms": ms,
                         "scatterings_per_s": events / (ms / 1e3), "gpu_launches": launches}

    # the surrogate network, trained on the GPU by the library's own kernels (untimed set-up)
    trainer = mc.Model(specs[0][0], device=dev, precision="mixed")
    vloss = trainer.surrogate_train(n_train=1 << 18, steps=40000, batch=4096, lr=2e-3, seed=1)
    weights = trainer.surrogate_weights()
    del trainer

    for form, sur in (("batched_mixed", False), ("batched_mixed_surrogate", True)):
        ctxs = []
        for (p, g, _) in specs:
            m = mc.Model(p, device=dev, precision="mixed", surrogate=sur)
            if sur:
                m.surrogate_weights(weights)
            m.set_grid(g)
            ctxs.append(m)
        t0 = time.perf_counter()
        mc.run_batch(ctxs, ns, seeds, autotune=True, graph=True, stream=stream)   # tune + capture
        t_setup = time.perf_counter() - t0
        flush.zero_()
        e0.record(stream)
        st = mc.run_batch(ctxs, ns, seeds, autotune=True, graph=True, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1)
        u = st["n_emit"] + st["n_child"]
        errs = [spectrum_error(c.spectrum_sums(), r) for c, r in zip(ctxs, ref)]
        lum = [e[0] for e in errs]
        nb, nok = sum(e[1] for e in errs), sum(e[2] for e in errs)
        fp64_flops = (FLOP_STEP_GRID_MIXED * st["n_steps_grid"] + FLOP_ITER * st["n_iters"]
                      + FLOP_STEP_FREE * (st["n_steps"] - st["n_steps_grid"]) + FLOP_EVENT * st["n_events"]
                      + FLOP_EMIT * st["n_emit"])
        kern_s = st["transport_ms"] / 1e3
        r = {"value": u / (bms / 1e3), "unit": UNIT, "superphotons": u, "ms": bms,
             "speedup_vs_plain_fp64": (u / (bms / 1e3)) / out["plain_fp64"]["value"],
             "scatterings_per_s": st["n_events"] / (bms / 1e3),
             "spectrum_error": {"total_luminosity_rel_max": max(lum), "total_luminosity_rel_median": float(np.median(lum)),
                                "bins_within_max_1pct_3sigma": nok / max(nb, 1), "bins_compared": nb,
                                "within_1pct": bool(max(lum) <= 0.01)},
             "autotune": {"min_blocks_per_sm": st["batch_min_blocks"], "ctas": st["batch_ctas"],
                          "graph": bool(st["batch_graph"]), "tune_and_capture_s": t_setup},
             "gpu_launches": 1 + GEN_LAUNCHES * len(specs) + 1,
             "roofline": df_roofline(fp64_flops, kern_s, fp32_peak, fp64_peak,
                                     "k_batch (whole batched transport, one cooperative launch)")}
        if sur:
            tf = FLOP_SUR_EVAL * st["n_steps_grid"] / kern_s / 1e12
            r["surrogate"] = {"validation_loss": vloss, "tensor_achieved_tflops": tf, "bf16_peak_tflops": bf16_peak,
                              "tensor_frac": tf / bf16_peak if bf16_peak else None,
                              "evals": st["n_steps_grid"]}
        out[form] = r
        del ctxs
        torch.cuda.empty_cache()
    return out


def main():
    global N_S, TAUS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass (profiling runs)")
    ap.add_argument("--n-s", type=float, default=N_S, help="N_s per run (smaller cases for profiling)")
    ap.add_argument("--taus", default=",".join(str(t) for t in TAUS), help="comma-separated Thomson depths")
    ap.add_argument("--no-survey", action="store_true", help="skip the batched-survey form")
    ap.add_argument("--survey-scale", type=float, default=1.0, help="N_s multiplier of the survey form")
    args = ap.parse_args()
    N_S = args.n_s
    TAUS = tuple(float(t) for t in args.taus.split(","))

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2602_13198_gb300 import synth

    cores = os.cpu_count() or 1
    if args.impl == "reference":
        # the reference arm is the CPU oracle (there is no reference implementation to install):
        # rank 0 times it on the host cores, a bounded sample of the same workload per step
        if rank != 0:
            return
        import oracle
        oracle.build()
        models = [synth.scattering_sphere(t) for t in TAUS]
        for w in range(args.warmup):
            p, g = models[w % len(models)]
            oracle_rate(p, g, 1, 2.0, cores, first_n=64)
        units, secs = 0, 0.0
        samples = []
        for k in range(args.steps):
            p, g = models[k % len(models)]
            seed = 1 + (k // len(models)) % 4
            rate, u, dt, n = oracle_rate(p, g, seed, 12.0, cores)
            units += u
            secs += dt
            samples.append(n)
        v = units / secs
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": WORKLOAD, "n_s_per_run": N_S},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": "first %s primaries (and their scattered descendants) of each step's job" % samples},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2602_13198_gb300 import build, mc
    build.build()
    dev = torch.cuda.current_device()
    models, ctxs = [], []
    for t in TAUS:
        p, g = synth.scattering_sphere(t)
        m = mc.Model(p, device=dev, precision=args.precision)
        m.set_grid(g)
        models.append((p, g))
        ctxs.append(m)
    fp64_peak = mc.fma_peak(dev, True)
    fp32_peak = mc.fma_peak(dev, False)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    nt = len(TAUS)

    def one(k, ctx_seed_offset=0):
        i = k % nt
        seed = 1 + (k // nt) % 4 + 1000 * rank + ctx_seed_offset
        return ctxs[i].run(N_S, seed, stream=stream)

    for w in range(args.warmup):
        one(w)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(dev)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        stats.append(one(k))
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    units = sum(s["n_emit"] + s["n_child"] for s in stats)
    t_transport = sum(s["transport_ms"] for s in stats) / 1e3
    launches = sum(s["transport_launches"] for s in stats)
    fgrid = FLOP_STEP_GRID if args.precision == "fp64" else FLOP_STEP_GRID_MIXED
    flops_grid = sum(fgrid * s["n_steps_grid"] + FLOP_ITER * s["n_iters_grid"] + FLOP_EVENT * s["n_events"]
                     for s in stats)
    flops = flops_grid + sum(FLOP_STEP_FREE * (s["n_steps"] - s["n_steps_grid"])
                             + FLOP_ITER * (s["n_iters"] - s["n_iters_grid"]) + FLOP_EMIT * s["n_emit"] for s in stats)
    t_grid = sum(s["grid_ms"] for s in stats) / 1e3
    t_free = sum(s["free_ms"] for s in stats) / 1e3
    t_init = sum(s["init_ms"] for s in stats) / 1e3
    if dist:
        t = torch.tensor([dev_s, float(units)], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        dev_s_max, units_all = float(tmax[0]), float(t[1])
    else:
        dev_s_max, units_all = dev_s, float(units)
    value = units_all / dev_s_max

    # end to end through the public API with host buffers: grid H2D each step, spectrum D2H
    import numpy as np
    host_prims = []
    for p, g in models:
        hp = torch.from_numpy(np.ascontiguousarray(g["prim"])).pin_memory()
        host_prims.append(hp)
    e2e_units, t_e2e = 0, 1e-300
    torch.cuda.synchronize()
    for k in range(0 if args.no_e2e else args.steps):
        i = k % nt
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctxs[i].set_grid(models[i][1], prim=host_prims[i].numpy())
        s = ctxs[i].run(N_S, 1 + (k // nt) % 4 + 1000 * rank, stream=stream)
        spec = ctxs[i].spectrum()
        t_e2e += time.perf_counter() - t0
        e2e_units += s["n_emit"] + s["n_child"]
    h2d = int(host_prims[0].numel() * 8)
    d2h = int(ctxs[0].n_incl * ctxs[0].n_bins * 3 * 8)
    if dist:
        t = torch.tensor([t_e2e, float(e2e_units)], dtype=torch.float64, device="cuda")
        tm = t.clone()
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        e2e_value = float(t[1]) / float(tm[0])
    else:
        e2e_value = e2e_units / t_e2e

    achieved = flops_grid / t_grid / 1e12
    peak = fp64_peak / 1e12
    per_run = units / max(args.steps, 1)
    if args.precision == "mixed":
        roofline = df_roofline(flops_grid, t_grid, fp32_peak, fp64_peak, "k_push<in-grid> (mixed, double-float geodesic)")
        roofline.update({"traffic": None, "phase_s": {"init": t_init, "in_grid": t_grid, "free": t_free}})
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": TRAFFIC_B_PER_PH_FP64 * per_run if TRAFFIC_B_PER_PH_FP64 else None,
                    "traffic_note": "bytes of the first in-grid launch of a run (it carries every primary): ncu DRAM "
                                    "read+write per superphoton at N_s=1e6 x superphotons per run",
                    "kernel": "k_push<in-grid> (%s): dominant kernel, %.0f%% of transport time"
                              % (args.precision, 100 * t_grid / max(t_transport, 1e-30)),
                    "peak_source": "measured: project FP64 FMA-chain microbenchmark on this GPU (mc_fma_peak)",
                    "fp32_peak_tflops": fp32_peak / 1e12,
                    "phase_s": {"init": t_init, "in_grid": t_grid, "free": t_free},
                    "transport_achieved_tflops": flops / t_transport / 1e12}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        p, g = models[min(2, nt - 1)]
        rate, u, dt, n = oracle_rate(p, g, 1, 15.0, cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "first %d primaries (+ scattered descendants, %d superphotons) of the tau_T=1e-2 seed-1 job, "
                         "%.1f s" % (n, u, dt)}
    survey = None
    if world == 1 and not args.no_survey:
        bf16 = None
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                bf16 = json.load(f).get("bf16_tflops")
        except Exception:
            bf16 = None
        survey = survey_forms(args, dev, stream, flush, fp64_peak, fp32_peak, bf16)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * dev_s_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "form": "plain FP64" if args.precision == "fp64" else "mixed FP64/FP32",
                           "n_s_per_run": N_S, "grid": [1024, 128, 1], "l2": "flushed (256 MiB write) between timed steps",
                           "parallelism": "replicas (independent jobs per rank)" if world > 1 else "single GPU"},
                "clocks": clocks,
                "e2e": None if args.no_e2e else {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                                                  "d2h_bytes_per_step": d2h},
                "roofline": roofline, "cpu_baseline": cpu, "survey": survey,
                "gpu_launches": int(launches + GEN_LAUNCHES * args.steps),
                "detail": {"superphotons": units, "scattered": sum(s["n_child"] for s in stats),
                           "steps_per_superphoton": sum(s["n_steps"] for s in stats) / max(units, 1),
                           "iters_per_step": sum(s["n_iters"] for s in stats) / max(1, sum(s["n_steps"] for s in stats)),
                           "step_ms": step_ms, "wall_s": t_wall,
                           "generate_ms": [s["generate_ms"] for s in stats],
                           "scatterings_per_s": sum(s["n_events"] for s in stats) / dev_s}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
