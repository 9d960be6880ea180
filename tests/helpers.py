"""Shared helpers for the parity tests: running the CUDA path and the oracle on the same
seeded inputs and comparing per-superphoton end states matched by random-stream id."""
import math

import numpy as np
import pytest

from paper_2602_13198_gb300 import synth

ME, CL = 9.1093837015e-28, 2.99792458e10


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def gpu_model(params, grid, precision="fp64", prim=None):
    from paper_2602_13198_gb300 import build, mc
    build.build()
    m = mc.Model(params, device=0, precision=precision)
    m.set_grid(grid, prim=prim)
    return m


def oracle_model(params, grid):
    import oracle
    return oracle.Model(params, grid)


def compare_logs(lg, lo, rtol=1e-9):
    """Match end states by stream id.  Returns a dict with the number matched, the ids whose
    discrete history differs (status, step count or event count: a decision flip), and the
    largest relative deviation of position, wavevector and weight over the others."""
    dg = {int(r["id"]): r for r in lg}
    do = {int(r["id"]): r for r in lo}
    common = sorted(set(dg) & set(do))
    only = (set(dg) ^ set(do))
    flips = []
    worst = {"X": 0.0, "K": 0.0, "w": 0.0}
    for i in common:
        a, b = dg[i], do[i]
        if a["status"] != b["status"] or a["nsteps"] != b["nsteps"] or a["nev"] != b["nev"] or a["gen"] != b["gen"]:
            flips.append(i)
            continue
        sx = np.maximum(np.maximum(np.abs(a["X"]), np.abs(b["X"])), 1.0)
        worst["X"] = max(worst["X"], float(np.max(np.abs(a["X"] - b["X"]) / sx)))
        sk = max(float(np.max(np.abs(a["K"]))), float(np.max(np.abs(b["K"]))), 1e-300)
        worst["K"] = max(worst["K"], float(np.max(np.abs(a["K"] - b["K"])) / sk))
        sw = max(abs(a["w"]), abs(b["w"]), 1e-300)
        worst["w"] = max(worst["w"], abs(a["w"] - b["w"]) / sw)
    return {"n": len(common), "flips": flips, "unmatched": len(only), "worst": worst}


def spectra_agree(sg, so, frac=0.01, nsig=3.0, min_count=1):
    """Per bin: |L_gpu - L_oracle| <= max(frac * L_oracle, nsig * sigma) with sigma the combined
    Monte Carlo standard error (bins with fewer than min_count superphotons on both sides skipped)."""
    a, b = sg[..., 0], so[..., 0]
    sig = np.sqrt(sg[..., 1] + so[..., 1])
    n = np.maximum(sg[..., 2], so[..., 2])
    sel = n >= min_count
    bad = sel & (np.abs(a - b) > np.maximum(frac * np.abs(b), nsig * sig))
    return not bad.any(), np.argwhere(bad)


def flat_sphere(n1=256, n2=32, **kw):
    return synth.sphere("flat", R=1.0, ne=1e13, thetae=100.0, B_gauss=1.0, n1=n1, n2=n2, r_record=3000.0, **kw)


requires_gpu = pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")
