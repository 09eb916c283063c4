"""The multi-rank bookkeeping on two gloo ranks (CPU): whole-job throughput
over the slowest rank, particle totals, the sum of per-rank gradients, and
distinct per-rank seeds."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2007_14401_gb300 import multi
        n_local = 1000 * (rank + 1)            # ranks may hold different counts
        ms_local = 10.0 + 5.0 * rank           # rank 1 is the slower one
        rate, ms, total = multi.whole_job_rate(n_local, 4, ms_local)
        g = torch.full((64,), float(rank + 1), dtype=torch.float64)
        multi.sum_over_ranks(g)
        seeds = [torch.tensor([multi.rank_seed(rank)]) for _ in range(world)]
        dist.all_gather(seeds, torch.tensor([multi.rank_seed(rank)]))
        out[rank] = (rate, ms, total, float(g[0]), float(g[-1]), [int(s) for s in seeds])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn")
    for r in range(world):
        rate, ms, total, g0, g1, seeds = out[r]
        assert ms == 15.0 and total == 3000
        assert rate == pytest.approx(3000 * 4 / 15e-3)
        assert g0 == g1 == 3.0
        assert seeds == [1, 2]


def test_single_process_is_identity():
    from paper_2007_14401_gb300 import multi
    rate, ms, total = multi.whole_job_rate(500, 2, 4.0)
    assert (ms, total) == (4.0, 500) and rate == pytest.approx(500 * 2 / 4e-3)
    x = torch.ones(3)
    assert torch.equal(multi.sum_over_ranks(x), torch.ones(3))
