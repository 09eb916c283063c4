"""The multi-rank bookkeeping on two gloo ranks (CPU): whole-job throughput
over the slowest rank, particle totals, the sum of per-rank gradients,
distinct per-rank seeds, and the push statistics reduced over ranks that
each push their own shard of one particle set."""
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


def _shard_worker(rank, world, port, out):
    """Each rank pushes its contiguous shard of one particle set with the
    FP64 oracle and reduces the statistics over the ranks."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        from paper_2007_14401_gb300 import inputs, multi
        from tests.helpers import oracle_field, oracle_params
        fields, st, p = inputs.harris_2d(n_per_species=96, seed=5)
        n = st["flags"].size
        lo, hi = n * rank // world, n * (rank + 1) // world
        shard = inputs.subset(st, np.arange(lo, hi))
        of, op = oracle_field(fields), oracle_params(p)
        per_call = []
        for _ in range(3):                    # one reduction per push call
            s = O.push_sr(shard, of, op, 4, nthreads=1)
            per_call.append(multi.reduce_stats(s))
        out[rank] = per_call
    finally:
        dist.destroy_process_group()


def test_stats_reduced_over_rank_shards_equal_one_process(orc):
    """Two gloo ranks each push half of the Harris particle set (the oracle
    per rank, the four q/m species spread over both); the statistics reduced
    over the ranks after every call equal those of one process pushing the
    whole set."""
    from paper_2007_14401_gb300 import inputs
    from tests.helpers import oracle_field, oracle_params
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shard_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn")
    fields, st, p = inputs.harris_2d(n_per_species=96, seed=5)
    of, op = oracle_field(fields), oracle_params(p)
    whole = [orc.push_sr(st, of, op, 4, nthreads=1) for _ in range(3)]
    for r in range(world):
        for got, ref in zip(out[r], whole):
            for k, v in ref.items():
                if k == "sum_ekin":
                    assert got[k] == pytest.approx(v, rel=1e-12)
                else:
                    assert got[k] == v, k
    assert whole[0]["n_gca"] > 0 and whole[0]["n_boris"] > 0
    assert out[0] == out[1]


def test_reduce_stats_single_process_is_identity():
    from paper_2007_14401_gb300 import multi
    s = {"n_boris": 3, "n_gca": 5, "n_to_gca": 1, "n_to_boris": 0, "n_nonconv": 0,
         "n_gcafail": 0, "n_nonfinite": 0, "sum_iter": 15, "max_iter": 4, "sum_ekin": 0.25,
         "n_exited": 2}
    assert multi.reduce_stats(s) == s


def _current_worker(rank, world, port, out):
    """Each rank pushes its contiguous shard with the oracle, depositing its
    particles' current, and sums the current over the ranks."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        from paper_2007_14401_gb300 import inputs, multi
        from tests.helpers import oracle_field, oracle_params
        fields, st, p = inputs.reconnection_2d(nx=32, ny=16, n_particles=301, seed=6,
                                               omega_dt_max=50.0)
        n = st["flags"].size
        lo, hi = n * rank // world, n * (rank + 1) // world
        shard = inputs.subset(st, np.arange(lo, hi))
        cur = O.Current(fields["E"][0].shape, q=(-1.0, 1.0))
        O.push_sr(shard, oracle_field(fields), oracle_params(p), 2, nthreads=1, current=cur)
        J = torch.as_tensor(np.stack(cur.J))
        out[rank] = multi.reduce_current(J).numpy()
    finally:
        dist.destroy_process_group()


def test_current_reduced_over_rank_shards_equals_one_process(orc):
    """Two gloo ranks deposit the current of their halves of one particle set
    (two pushes each); after reduce_current both hold the current one process
    deposits for the whole set, to rounding."""
    from paper_2007_14401_gb300 import inputs
    from tests.helpers import oracle_field, oracle_params
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_current_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn")
    fields, st, p = inputs.reconnection_2d(nx=32, ny=16, n_particles=301, seed=6,
                                           omega_dt_max=50.0)
    cur = orc.Current(fields["E"][0].shape, q=(-1.0, 1.0))
    orc.push_sr(st, oracle_field(fields), oracle_params(p), 2, nthreads=1, current=cur)
    want = np.stack(cur.J)
    scale = np.abs(np.stack(cur.Jabs)).max()
    for r in range(world):
        assert np.abs(out[r] - want).max() <= 1e-13 * scale
    assert np.array_equal(out[0], out[1]) and np.abs(want).max() > 0


def test_reduce_current_single_process_is_identity():
    from paper_2007_14401_gb300 import multi
    J = torch.arange(12.0).reshape(3, 2, 2)
    assert torch.equal(multi.reduce_current(J.clone()), J)
