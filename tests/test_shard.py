"""Sharding one camera across ranks: partition logic, a 2-rank gloo run on
CPU (FP64 oracle as the per-rank compute) and, on a GPU, virtual ranks whose
partial sums add up to the single-call result."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1909_04573_gb300 import shard


@pytest.mark.parametrize("m,d,world", [(64, 8, 2), (37, 8, 2), (37, 8, 3), (10, 10, 4), (100, 1, 3), (5, 2, 8)])
def test_partition_covers_whole_groups_once(m, d, world):
    parts = shard.partition_groups(m, d, world)
    assert len(parts) == world
    covered = []
    for f0, f1 in parts:
        assert f0 <= f1
        assert f0 % d == 0 or f0 == m           # runs start at group boundaries
        assert f1 % d == 0 or f1 == m
        covered.extend(range(f0, f1))
    assert covered == list(range(m))             # contiguous, disjoint, complete
    sizes = [(f1 - f0 + d - 1) // d for f0, f1 in parts]
    assert max(sizes) - min(sizes) <= 1           # balanced to one group


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, frames, d, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        m, H, W, C = frames.shape
        num = torch.zeros((C, H, W), dtype=torch.float64)
        den = torch.zeros_like(num)

        def acc(fr, dd, nm, dn):
            n_, d_ = O.fingerprint_accumulate(fr, dd)
            nm += torch.from_numpy(n_)
            dn += torch.from_numpy(d_)

        shard.accumulate_sharded(acc, frames, d, num, den, rank, world)
        out[rank] = (num.numpy(), den.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sum_equals_single_process():
    import oracle as O
    rng = np.random.default_rng(3)
    frames = rng.integers(0, 256, size=(21, 32, 40, 1), dtype=np.uint8)
    d, world = 4, 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), frames, d, out), nprocs=world, join=True,
                       start_method="spawn")
    num, den = O.fingerprint_accumulate(frames, d)
    for r in range(world):
        np.testing.assert_allclose(out[r][0], num, rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(out[r][1], den, rtol=1e-12)


@pytest.mark.gpu
def test_virtual_ranks_on_one_gpu_sum_to_single_call():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04573_gb300 import prnu as P
    from paper_1909_04573_gb300 import synth
    ctx = P.Context(0)
    try:
        fr = synth.frames(synth.Camera(H=96, W=128, C=3, camera_id=12), 43, device="cuda", drift_px=1.0)
        full_n = torch.zeros((3, 96, 128), device="cuda")
        full_d = torch.zeros_like(full_n)
        ctx.fingerprint_accumulate(fr, 5, full_n, full_d)
        sum_n = torch.zeros_like(full_n)
        sum_d = torch.zeros_like(full_n)
        world = 3
        for rank in range(world):
            n = torch.zeros_like(full_n)
            dd = torch.zeros_like(full_n)
            shard.accumulate_sharded(lambda f, d_, a, b: ctx.fingerprint_accumulate(f, d_, a, b), fr, 5, n, dd,
                                     rank, world, reduce=False)
            sum_n += n      # the host-side sum stands in for the all-reduce
            sum_d += dd
        torch.cuda.synchronize()
        assert float((sum_n - full_n).norm() / full_n.norm()) <= 1e-6
        assert float((sum_d - full_d).norm() / full_d.norm()) <= 1e-6
    finally:
        ctx.close()
