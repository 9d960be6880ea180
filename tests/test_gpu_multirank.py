"""The sharded job through the CUDA path: two gloo ranks (two processes sharing the one GPU), each
running its contiguous uid shard of the same job with mc_run and summing counters and spectrum
accumulators with mc.run_sharded.  The ranks' kernels never wait on one another; the only exchange
is the host-side allreduce.  The result equals the whole job run in one process: counters exactly,
spectrum sums to summation-order rounding, and the whole job equals the oracle's spectrum."""
import os
import socket
import tempfile

import numpy as np
import pytest

from helpers import oracle_model, requires_gpu, spectra_agree
from paper_2602_13198_gb300 import synth

pytestmark = [pytest.mark.gpu, requires_gpu]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name):
    if name == "ks_scatter":
        return synth.scattering_sphere(1e-1, n1=256, n2=64), 5e4, 4
    return synth.torus(a=-0.5, n1=96, n2=48, R_high=1.0, M_unit=1e18, seed=61), 3e4, 5


def _rank_main(rank, world, port, name, precision, out):
    import torch.distributed as dist

    from paper_2602_13198_gb300 import mc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        (p, g), n_s, seed = _case(name)
        m = mc.Model(p, device=0, precision=precision)
        m.set_grid(g)
        stats, sums = mc.run_sharded(m, n_s, seed)
        if rank == 0:
            np.savez(out, sums=sums, **{k: stats[k] for k in mc.SUMMED_STATS + ("n_total",)})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,precision", [("ks_scatter", "fp64"), ("retro_torus", "fp64"), ("retro_torus", "mixed")])
def test_two_gloo_ranks_on_the_cuda_path_equal_the_whole_job(name, precision):
    import torch.multiprocessing as tmp

    from paper_2602_13198_gb300 import build, mc
    build.build()
    (p, g), n_s, seed = _case(name)
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "r.npz")
        tmp.start_processes(_rank_main, args=(2, _free_port(), name, precision, out), nprocs=2, join=True,
                            start_method="spawn")
        got = np.load(out)
    m = mc.Model(p, device=0, precision=precision)
    m.set_grid(g)
    whole = m.run(n_s, seed)
    ws = m.spectrum_sums()
    assert int(got["n_total"]) == whole["n_total"]
    for k in ("n_emit", "n_child", "n_rec", "n_abs", "n_capt", "n_steps", "n_iters", "n_events", "n_steps_grid"):
        assert int(got[k]) == whole[k], k
    assert whole["n_child"] > 0
    assert np.array_equal(got["sums"][..., 2], ws[..., 2])
    assert np.allclose(got["sums"], ws, rtol=1e-11, atol=0)
    if precision == "fp64":
        om = oracle_model(p, g)
        om.prepare(n_s, seed)
        ok, bad = spectra_agree(got["sums"], om.run()["spec"])
        assert ok, bad
