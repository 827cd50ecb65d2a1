"""World-size-2 run of the bench's multi-rank host logic on CPU (gloo): each
rank builds its own seeded batch of the same configuration (weak scaling, no
data exchange), and the whole-job figures are the slowest rank's time and the
sum of the ranks' work."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    wl = bench.make_workload(2, rank)
    bt = wl.batch
    ms = 1.0 + 0.5 * rank  # rank 1 is the slow one
    out = bench.reduce_over_ranks(ms, bt.n_bandflux(), bt.n_par, "cpu")
    q.put((rank, out, bt.n_bandflux(), bt.n_par, float(bt.z[:8].sum()), int(bt.obs_off[-1])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_supernovae_and_reduce_max_time_sum_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, out0, nbf0, npar0, zs0, nobs0), (r1, out1, nbf1, npar1, zs1, nobs1) = res
    assert out0 == out1  # every rank sees the same whole-job figures
    ms_max, nbf_all, npar_all = out0
    assert ms_max == 1.5
    assert nbf_all == nbf0 + nbf1 and npar_all == npar0 + npar1
    assert npar0 == npar1 == 1000  # same configuration shape on every rank
    assert zs0 != zs1 and nobs0 != nobs1  # but each rank owns different supernovae
