"""Partial cells of the sphere set-up (section 4.1): inside fractions in steps of 1/5 only at the
edge, and an emitting volume (the code's midpoint-rule zone volumes x fraction) that approaches
4 pi R^3 / 3 more closely than the abrupt edge of the same grid."""
import math

import numpy as np

from paper_2602_13198_gb300 import synth


def emitting_volume(n1, partial, n2=128):
    p, g = synth.sphere("flat", R=1.0, ne=1e13, thetae=100.0, B_gauss=1.0, n1=n1, n2=n2, r_out=1e4,
                        partial=partial)
    X1, X2, _ = synth._zone_centres(g)
    vol = np.exp(3 * X1) * np.sin(math.pi * X2) * math.pi * g["dx1"] * g["dx2"] * g["dx3"]
    return float((vol * g["prim"][0]).sum()), g


def test_fractions_only_at_the_edge():
    _, g = emitting_volume(32000, 5, n2=2)
    f = g["prim"][0]
    assert set(np.round(np.unique(f) * 5).astype(int)) <= {0, 1, 2, 3, 4, 5}
    edge = (f > 0) & (f < 1)
    X1, _, _ = synth._zone_centres(g)
    assert np.all(np.abs(X1[edge]) < g["dx1"])          # ln R = 0 lies in those zones
    assert np.all(f[X1 < -g["dx1"]] == 1.0) and np.all(f[X1 > g["dx1"]] == 0.0)


def test_partial_cells_cut_the_volume_bias():
    exact = 4.0 * math.pi / 3.0
    v_abrupt, _ = emitting_volume(8192, 0)
    v_part, _ = emitting_volume(32000, 5)
    # 128 polar cells: the midpoint rule in theta alone is 2.5e-5 low
    assert abs(v_part / exact - 1.0) < 2e-4
    assert abs(v_part / exact - 1.0) < 0.2 * abs(v_abrupt / exact - 1.0)
