"""Multi-rank path on the CPU (gloo, world size 2): shot partition, max-over-ranks timing
and the stacked-gradient sum used when one survey is split across GPUs."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2201_06914_gb300.dist import shot_range


def test_shot_range_partition():
    for total in (1, 7, 64, 65):
        for world in (1, 2, 3, 8):
            got = [s for r in range(world) for s in shot_range(total, r, world)]
            assert got == list(range(total))
            sizes = [len(shot_range(total, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2201_06914_gb300.dist import max_over_ranks, shot_range, sum_image
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shot_range(10, rank, world)
        # each rank "images" its own shots: a per-shot image equal to the shot index
        g = torch.zeros(5, dtype=torch.float64)
        for s in mine:
            g += s
        sum_image(g)
        t = max_over_ranks(0.5 + rank)
        q.put((rank, list(mine), g.tolist(), t))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] + out[1][1] == list(range(10))
    for rank, _, g, t in out:
        assert np.allclose(g, sum(range(10)))   # stacked over both ranks
        assert t == 1.5                          # slowest rank
