"""mc_zone_counts_noalloc: zone counts for callers that cannot allocate device memory (a stream
under graph capture, an allocator callback, an application owning all device memory).  Its
scratch is a fixed static device array; the tests check it against the counts of the regular
entry points (mc_run, then mc_get_zone_counts) on two calls in a row, for thermal, kappa and
bremsstrahlung models (the last two have per-zone arrays of their own, which the call rebuilds in
its scratch), that a non-finite zone state makes the device total -1 (mc_run fails there), and that
grids above the stated maximum are refused.  Collected last so that a failure here stops a -x run
only after every other test has run."""
import numpy as np
import pytest

from helpers import requires_gpu
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]


def _buffers(nz):
    import torch
    return (torch.zeros(nz, dtype=torch.int64, device="cuda"), torch.zeros(nz, dtype=torch.int64, device="cuda"),
            torch.zeros(1, dtype=torch.int64, device="cuda"))


def _check_against_run(m, jobs):
    import torch
    counts, start, total = _buffers(m.nz)
    for n_s, seed in jobs:
        st = m.run(n_s, seed)
        ref = m.zone_counts()
        spec_before = m.spectrum_sums()
        for _ in range(2):                        # two calls in a row reuse the same scratch
            counts.fill_(-1)
            start.fill_(-1)
            total.fill_(-1)
            m.zone_counts_noalloc(n_s, seed, counts, start, total)
            torch.cuda.synchronize()
            c = counts.cpu().numpy()
            assert np.array_equal(c, ref)         # integer counts: bit-exact
            s = start.cpu().numpy()
            assert s[0] == 0 and np.array_equal(s[1:], np.cumsum(ref)[:-1])
            assert int(total.item()) == int(ref.sum()) == st["n_total"]
        # the context's own results are left as the run wrote them
        assert np.array_equal(m.spectrum_sums(), spec_before)
        assert np.array_equal(m.zone_counts(), ref)


def test_noalloc_counts_match_regular_entry_points():
    from paper_2602_13198_gb300 import build, mc
    build.build()
    p, g = synth.scattering_sphere(1e-2)          # 1024 x 128 = 131072 zones, the supported maximum
    m = mc.Model(p)
    m.set_grid(g)
    _check_against_run(m, ((1e6, 3), (2e5, 8)))


@pytest.mark.parametrize("kind", ["kappa", "brems"])
def test_noalloc_counts_kappa_and_bremsstrahlung(kind):
    from paper_2602_13198_gb300 import mc
    if kind == "kappa":
        p, g = synth.scattering_sphere(0.1, n1=256, n2=64, kappa=5.0)
    else:
        p, g = synth.scattering_sphere(1e-1, n1=64, n2=16)
        p = dict(p, brems=1)
    m = mc.Model(p)
    m.set_grid(g)
    _check_against_run(m, ((3e4, 5), (1e4, 6)))
    # a second run after the allocation-free calls still equals the first (context arrays untouched)
    st = m.run(3e4, 5)
    ref = m.zone_counts()
    counts, start, total = _buffers(m.nz)
    m.zone_counts_noalloc(3e4, 5, counts, start, total)
    assert np.array_equal(counts.cpu().numpy(), ref) and int(total.item()) == st["n_total"]


def test_noalloc_reports_non_finite_zone_state():
    import torch

    from paper_2602_13198_gb300 import mc
    p, g = synth.scattering_sphere(1e-2, n1=64, n2=16)
    prim = np.array(g["prim"], dtype=np.float64, copy=True)
    prim[2, 100] = 1e200                          # finite primitive, but b^2 overflows: |B| = inf
    g = dict(g, prim=prim)
    m = mc.Model(p)
    m.set_grid(g)
    with pytest.raises(mc.MCError) as e:
        m.run(1e4, 1)
    assert e.value.code == -6                     # MC_ERR_NAN_INPUT
    counts, start, total = _buffers(m.nz)
    for _ in range(2):
        total.fill_(7)
        m.zone_counts_noalloc(1e4, 1, counts, start, total)
        torch.cuda.synchronize()
        assert int(total.item()) == -1
    # the scratch recovers on the next finite model
    p2, g2 = synth.scattering_sphere(1e-2, n1=64, n2=16)
    m2 = mc.Model(p2)
    m2.set_grid(g2)
    _check_against_run(m2, ((1e4, 1),))


def test_noalloc_rejects_grids_above_the_limit():
    import torch

    from paper_2602_13198_gb300 import mc
    p, g = synth.scattering_sphere(1e-2, n1=1025, n2=128)
    m = mc.Model(p)
    m.set_grid(g)
    buf = torch.zeros(m.nz, dtype=torch.int64, device="cuda")
    tot = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(mc.MCError) as e:
        m.zone_counts_noalloc(1e5, 1, buf, buf.clone(), tot)
    assert e.value.code == -7
