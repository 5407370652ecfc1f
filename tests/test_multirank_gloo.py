"""The multi-GPU path's host logic on CPU with two gloo ranks (127.0.0.1).

Channels are independent end to end, so N GPUs run N independent bands of
channels (weak scaling) and the only collective is the max over ranks of the
timed region.  Two spawned ranks each draw their own band (seed offset by the
rank), compute V^unique and the subset V^reduced of it with the oracle, and
reduce their (rank-dependent) step times.  Rank 0 checks that the gathered
bands equal what one process computes for the same seeds, that the bands
differ between ranks, that the time reduction is the max, and that the job
rate counts every rank's units over the slowest rank's time.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2005_03060_gb300 import shard, synth

L, C, T, BASE_SEED = 4, 2, 64, 11


def _band(orc, rank):
    from oracle import select as osel
    volt, gains, _ = synth.make_voltages(shard.rank_seed(BASE_SEED, rank), L, C, T, n_src=3)
    v = volt.numpy().astype(np.complex128)
    g = gains.numpy().astype(np.complex128)
    sel = osel.subset(L, T)
    pt = sel.pair_type()
    vu = np.stack([orc.fx(v[c], g[c], L) for c in range(C)])
    vr = np.stack([orc.xengine_c64(v[c], sel.pair_i, sel.pair_j, sel.win_t0[pt], sel.win_t1[pt])
                   for c in range(C)])
    return vu, vr


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as orc
        vu, vr = _band(orc, rank)
        ms = shard.max_over_ranks(100.0 + 25.0 * rank)
        rate = shard.job_rate(C * T * L * L, world, ms)
        got = [None] * world
        dist.all_gather_object(got, (vu, vr, ms, rate))
        if rank == 0:
            torch.save(got, out)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_shard_channels(orc, tmp_path):
    world = 2
    out = str(tmp_path / "gathered.pt")
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    got = torch.load(out, weights_only=False)
    assert len(got) == world
    for rank, (vu, vr, ms, rate) in enumerate(got):
        vu1, vr1 = _band(orc, rank)
        np.testing.assert_array_equal(vu, vu1)   # sharding changes no channel's result
        np.testing.assert_array_equal(vr, vr1)
        assert ms == 125.0                        # max over ranks, the same on every rank
        assert rate == pytest.approx(world * C * T * L * L / 0.125)
    assert not np.allclose(got[0][0], got[1][0])  # the ranks hold different bands


def test_single_process_helpers():
    assert shard.rank_seed(7, 0) == 7 and shard.rank_seed(7, 3) == 7 + 3 * shard.RANK_SEED_STRIDE
    assert shard.max_over_ranks(3.5) == 3.5       # no process group: the value itself
    assert shard.job_rate(10.0, 1, 1000.0) == pytest.approx(10.0)
    with pytest.raises(ValueError):
        shard.job_rate(1.0, 1, 0.0)
    with pytest.raises(ValueError):
        shard.rank_seed(0, -1)
