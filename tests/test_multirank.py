"""Multi-rank host path on CPU (gloo, world size 2): each rank takes its contiguous uid shard of
one job, the counters and spectrum accumulators are summed with the library's allreduce helpers,
and the result equals the whole job run in one process (counts exactly, sums to rounding)."""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2602_13198_gb300 import mc, synth


@pytest.mark.parametrize("total,world", [(0, 2), (1, 2), (7, 2), (1000003, 2), (12, 5), (5, 8)])
def test_shard_bounds_partition_the_job(total, world):
    spans = [mc.shard_bounds(total, r, world) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == total
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert a1 == b0 and a0 <= a1
    assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cases():
    thin = synth.sphere("flat", R=1.0, ne=1e13, thetae=100.0, B_gauss=1.0, n1=64, n2=16, r_record=3000.0)
    scat = synth.scattering_sphere(1e-1, n1=64, n2=16)
    return {"flat_thin": (thin, 2e3, 3), "ks_scatter": (scat, 1e3, 4)}


def _rank_main(rank, world, port, name, out):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        (p, g), n_s, seed = _cases()[name]
        om = oracle.Model(p, g)
        tot = om.prepare(n_s, seed)
        u0, u1 = mc.shard_bounds(tot, rank, world)
        r = om.run(u0, u1, nthreads=1)
        st = dict(r["stats"], n_total=tot, n_steps_grid=0, n_iters_grid=0)
        stats = mc.allreduce_stats(st)
        sums = mc.allreduce_spectrum(r["spec"])
        if rank == 0:
            np.savez(out, sums=sums, **{k: stats[k] for k in mc.SUMMED_STATS + ("n_total",)})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["flat_thin", "ks_scatter"])
def test_two_gloo_ranks_equal_the_whole_job(name):
    import torch.multiprocessing as tmp
    import oracle
    (p, g), n_s, seed = _cases()[name]
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "r.npz")
        tmp.start_processes(_rank_main, args=(2, _free_port(), name, out), nprocs=2, join=True,
                            start_method="spawn")
        got = np.load(out)
        om = oracle.Model(p, g)
        tot = om.prepare(n_s, seed)
        whole = om.run(nthreads=1)
        assert int(got["n_total"]) == tot
        for k in ("n_emit", "n_child", "n_rec", "n_abs", "n_capt", "n_steps", "n_events"):
            assert int(got[k]) == whole["stats"][k], k
        assert np.array_equal(got["sums"][..., 2], whole["spec"][..., 2])
        assert np.allclose(got["sums"], whole["spec"], rtol=1e-12, atol=0)
        if name == "ks_scatter":
            assert whole["stats"]["n_child"] > 0
