"""Config-1 sphere (Schwarzschild, R = 10 M, Theta_e = 10, n_e = 1e13, B = 10 G, 1024 x 128 grid) on the
device against the deterministic thin-bin reference (redshift + capture rule): at the config's
N_s = 1e5 (seed 1) and, for a sharper check, at N_s = 1e7."""
import math

import numpy as np
import pytest

import schwarzschild_sphere as ss
from helpers import gpu_model, requires_gpu
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]
ME, CL = 9.1093837015e-28, 2.99792458e10


@pytest.fixture(scope="module")
def reference():
    p, g = synth.sphere("ks")
    dlog = (p["lnu_hi"] - p["lnu_lo"]) / p["n_bins"]
    centres = p["lnu_lo"] + dlog * (np.arange(p["n_bins"]) + 0.5)
    b = np.where((centres > 13.4) & (centres < 15.0))[0]
    return p, g, b, ss.nuLnu_bins(p, 2.1, 10.0, 1e13, 10.0, 10.0, b)


@pytest.mark.parametrize("n_s,seed,min_count", [(1e5, 1, 100), (1e7, 2, 1000)])
def test_thin_bins_match_reference(reference, n_s, seed, min_count):
    p, g, b, ref = reference
    m = gpu_model(p, g)
    m.run(n_s, seed)
    S = m.spectrum_sums()[0]
    dln = (p["lnu_hi"] - p["lnu_lo"]) / p["n_bins"] * math.log(10)
    nuL = S[b, 0] * ME * CL * CL / dln
    sig = np.sqrt(S[b, 1]) * ME * CL * CL / dln
    sel = S[b, 2] >= min_count
    assert sel.sum() >= 10
    rel = nuL[sel] / ref[sel] - 1.0
    z = (nuL[sel] - ref[sel]) / sig[sel]
    print("N_s %.0e: %d thin bins, max |rel| %.2e, mean z %.2f" % (n_s, sel.sum(), np.abs(rel).max(), z.mean()))
    assert np.all((np.abs(rel) < 0.01) | (np.abs(z) < 4.0)), (rel, z)
    assert abs(np.mean(z)) < 3.0 / math.sqrt(sel.sum())
