"""The N > 1 host path of bench.py on CPU: two gloo ranks, each with its own frames.

Frames are independent, so ranks share no data on the decode path; the only
cross-rank steps are the timing (slowest rank) and the failure counts.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        x, y, e = bench.rank_inputs(4, rank)
        digest = torch.tensor([int(x[:, :4].astype(np.uint64).sum() % (2**31))], dtype=torch.int64)
        gathered = [torch.zeros_like(digest) for _ in range(world)]
        dist.all_gather(gathered, digest)
        ms, ms_e2e, fails, und = bench.reduce_over_ranks(dist, "cpu", 10.0 + rank, 20.0 - rank, rank, 1)
        out[rank] = (ms, ms_e2e, fails, und, [int(g) for g in gathered], bench.job_mbps(4, world, ms))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_frames_and_take_the_slowest_time():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, ms_e2e, fails, und, digests, mbps = res[rank]
        assert ms == 11.0 and ms_e2e == 20.0  # max over ranks
        assert fails == 1 and und == 2        # sums over ranks
        assert digests[0] != digests[1]      # each rank decodes different frames
        assert mbps == pytest.approx(4 * 65536 * 2 / 0.011 / 1e6)


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, "cpu", 3.0, 4.0, 1, 0) == (3.0, 4.0, 1, 0)
