"""Multi-rank bookkeeping: one process per GPU, particles sharded by rank.

Test particles in static fields do not interact, so the push exchanges
nothing between ranks.  What crosses ranks is bookkeeping: the step time (the
whole job is as slow as its slowest rank: max), the particle count (sum),
the push statistics (counters and the kinetic-energy sum: sum; the largest
fixed-point iteration count: max), and, after an adjoint sweep, the gradients
with respect to shared inputs such as the field-mode amplitudes (sum).  With
current deposition (the PiC coupling) there is one real exchange per step:
every rank deposits its own particles' current on its replica of the grid,
and the field solve needs their sum (reduce_current).  Each function is a
no-op reduction when no process group is initialised.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def _group_size() -> int:
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size()
    return 1


def rank_seed(rank: int) -> int:
    """Seed of rank's synthetic particles (distinct per rank, 1 on rank 0)."""
    return 1 + int(rank)


def whole_job_rate(n_local: int, steps: int, ms_local: float, device="cpu"):
    """Units processed by all ranks per second over the slowest rank's time.
    Returns (rate, max ms, total units)."""
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    n = torch.tensor([float(n_local)], dtype=torch.float64, device=device)
    if _group_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    total = int(round(n.item()))
    return total * steps / (ms * 1e-3), ms, total


def sum_over_ranks(x: torch.Tensor) -> torch.Tensor:
    """In-place sum over ranks (e.g. dL/da_m of each rank's particles)."""
    if _group_size() > 1:
        dist.all_reduce(x, op=dist.ReduceOp.SUM)
    return x


# gcb_stats fields summed over ranks (the rest: max_iter, a maximum)
STATS_SUM = ("n_boris", "n_gca", "n_to_gca", "n_to_boris", "n_nonconv", "n_gcafail",
             "n_nonfinite", "sum_iter", "sum_ekin", "n_exited")


def reduce_stats(stats: dict, device="cpu") -> dict:
    """Whole-job statistics of one push call from each rank's: one SUM
    allreduce of the counters and the kinetic-energy sum (float64, exact for
    counts below 2^53) and one MAX allreduce of max_iter.  Returns a new dict
    with the same keys; the identity without a process group."""
    s = torch.tensor([float(stats[k]) for k in STATS_SUM], dtype=torch.float64, device=device)
    m = torch.tensor([int(stats["max_iter"])], dtype=torch.int64, device=device)
    if _group_size() > 1:
        dist.all_reduce(s, op=dist.ReduceOp.SUM)
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
    out = {k: (float(v) if k == "sum_ekin" else int(round(float(v))))
           for k, v in zip(STATS_SUM, s.tolist())}
    out["max_iter"] = int(m.item())
    return {k: out[k] for k in stats}


def reduce_current(J: torch.Tensor) -> torch.Tensor:
    """In-place sum over ranks of each rank's deposited current (one SUM
    allreduce of the whole grid, 3 x nodes values): afterwards every rank
    holds the current of all particles, as the field solve of the next PiC
    step needs.  The identity without a process group."""
    if _group_size() > 1:
        dist.all_reduce(J, op=dist.ReduceOp.SUM)
    return J
