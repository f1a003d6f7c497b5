"""The multi-GPU path is replicas only: every rank runs its own walkers and Philox stream,
and the only collective is one MAX all-reduce of the timing. Checked here with two gloo
ranks on the CPU: distinct per-rank streams (the oracle's first draws differ), the slowest
rank's time seen by both, and the whole-job rate."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist   # noqa: E402
import torch.multiprocessing as mp   # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    from oracle.philox import move_draws
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        philox_seed, pos_seed = bench.replica_seeds(rank)
        xi, u = move_draws(philox_seed, 0, 0, 0)
        pos0 = np.random.default_rng(pos_seed).uniform(0, 1, 3)
        local_ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, dist, device="cpu")
        rate = bench.whole_job_rate(world, 1000.0, ms / 1e3)
        out[rank] = (philox_seed, pos_seed, float(u), tuple(pos0), ms, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    (s0, p0, u0, x0, ms0, r0), (s1, p1, u1, x1, ms1, r1) = res[0], res[1]
    assert s0 != s1 and p0 != p1                        # independent streams
    assert u0 != u1 and x0 != x1
    assert ms0 == ms1 == 15.0                           # both see the slowest rank
    assert r0 == r1 == pytest.approx(2 * 1000.0 / 0.015)
