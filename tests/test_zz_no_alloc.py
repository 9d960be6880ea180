"""mc_zone_counts_noalloc: zone counts for callers that cannot allocate device memory (a stream
under graph capture, an allocator callback, an application owning all device memory).  Its
scratch is a fixed static device array; the test checks it against the counts of the regular
entry points (mc_run, then mc_get_zone_counts) on two calls in a row, and that grids above the
stated maximum are refused.  Collected last so that a failure here stops a -x run only after
every other test has run."""
import numpy as np
import pytest

from helpers import requires_gpu
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]


def test_noalloc_counts_match_regular_entry_points():
    import torch

    from paper_2602_13198_gb300 import build, mc
    build.build()
    p, g = synth.scattering_sphere(1e-2)          # 1024 x 128 = 131072 zones, the supported maximum
    m = mc.Model(p)
    m.set_grid(g)
    nz = m.nz
    counts = torch.zeros(nz, dtype=torch.int64, device="cuda")
    start = torch.zeros(nz, dtype=torch.int64, device="cuda")
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    for n_s, seed in ((1e6, 3), (2e5, 8)):
        st = m.run(n_s, seed)
        ref = m.zone_counts()
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
