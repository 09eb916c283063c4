"""Throughput of the coupled guiding-center / Boris push on one GB300.

Workload: the 2D reconnection-like field (double Harris sheet with a GEM-style
flux perturbation, 64 random-phase Fourier modes, E = -v_in x B) on a
2048 x 1024 periodic grid with float32 fields and precomputed float32
gradient grids, 2^24 Maxwell-Juttner positrons and electrons (theta = 1),
dt = 0.45, |q/m| with max Omega_C dt = 1e5: the mixed-precision path (float32
arithmetic, float32-pair positions).  A step is one pass of the whole push
over all particles (one kernel), state resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank pushes its own 2^24 particles (weak scaling, no
collective on the data path); rank 0 prints one JSON line.  --impl reference
times the FP64 CPU oracle on this machine's host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s"
NX, NY, NP = 2048, 1024, 1 << 24
SORT_EVERY = 8
SORT_TILE = (1, 1)
# algorithmic bytes per particle-step of the mixed path: state read + write
# (x as 2 float32 pairs 16 B, u 12 B, dxp 8 B, flags 1 B) and the field
# records (48 B per node) read once per step, divided over the particles.
STATE_B = 16 + 12 + 8 + 1
FIELD_B = NX * NY * 48
STATE_B64 = 16 + 24 + 16 + 1
FIELD_B64 = NX * NY * 96


def alg_bytes_per_launch(n, fp64=False):
    return (2 * (STATE_B64 if fp64 else STATE_B)) * n + (FIELD_B64 if fp64 else FIELD_B)


def workload_config(n_total, ngpu, sort_every=SORT_EVERY, sort_tile=SORT_TILE):
    return {"workload": f"2D double Harris + GEM + 64 modes, {NX}x{NY} grid, "
                        f"{n_total} particles, mixed FP32 (FP32-pair positions)",
            "grid": [NX, NY], "particles": n_total, "particles_per_gpu": n_total // ngpu,
            "dt": 0.45, "omega_c_dt_max": 1e5, "curvature": 1, "grad_mode": "grid",
            "gca_tol": 1e-7, "steps_per_call": 1, "sort_every": sort_every,
            "sort_tile": list(sort_tile),
            "l2": "inputs larger than L2 (particle state 620 MB per GPU)"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                       f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(fields, st, p, budget_s=15.0, n_sample=1 << 16):
    """The FP64 oracle (as it stands) on the host cores, on a bounded sample."""
    import oracle as O
    from paper_2007_14401_gb300 import inputs
    sub = inputs.subset(st, np.arange(n_sample))
    of = O.grid_field(fields["E"], fields["B"], fields["dx"], dB=fields["dB"])
    op = O.make_params(dt=p["dt"], qm=p["qm"], f_rho=p["f_rho"], f_E=p["f_E"], dl=p["dl"],
                       curvature=p["curvature"], grad_mode=p["grad_mode"],
                       max_iter=p["gca_max_iter"], tol=p["gca_tol"])
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t0 = time.perf_counter()
    O.push_sr(sub, of, op, 1, nthreads=cores)
    t1 = time.perf_counter() - t0
    steps = max(1, min(2000, int(budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    O.push_sr(sub, of, op, steps, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": n_sample * steps / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{n_sample} particles x {steps} steps of the same workload, FP64 "
                      f"oracle (C, OpenMP over particles), {dt:.1f} s"}


def run_reference(args, rank):
    if rank != 0:
        return 0
    from paper_2007_14401_gb300 import inputs
    fields, st, p = inputs.reconnection_2d(nx=NX, ny=NY, n_particles=1 << 14)
    import oracle as O
    O.build()
    of = O.grid_field(fields["E"], fields["B"], fields["dx"], dB=fields["dB"])
    op = O.make_params(dt=p["dt"], qm=p["qm"], curvature=1, grad_mode=1,
                       max_iter=p["gca_max_iter"], tol=p["gca_tol"])
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    n = st["flags"].size
    for _ in range(args.warmup):
        O.push_sr(st, of, op, 1, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.push_sr(st, of, op, 1, nthreads=cores)
    dt = time.perf_counter() - t0
    v = n * args.steps / dt
    line = {"metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": dict(workload_config(NP * args.gpus, args.gpus),
                           sample=f"{n} particles per step (bounded sample)"),
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"{n} particles x {args.steps} steps, FP64 oracle"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gcb", choices=["gcb", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sort-every", type=int, default=SORT_EVERY)
    ap.add_argument("--sort-tile", default=",".join(map(str, SORT_TILE)),
                    help="cells per sort tile, e.g. 2,2")
    ap.add_argument("--particles", type=int, default=NP,
                    help="particles per GPU (smaller cases for profiling only)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2007_14401_gb300 import gcb as G
    from paper_2007_14401_gb300 import inputs

    fields, st, p = inputs.reconnection_2d(nx=NX, ny=NY, n_particles=args.particles,
                                           seed=1 + rank)
    grid = G.Grid(fields, dtype="f32")
    ds = G.State.from_numpy(st, precision="mixed", pos_mode="pair")
    tile = tuple(int(v) for v in args.sort_tile.split(","))
    gp = G.make_params(p, sort_every=args.sort_every, sort_tile=tile)
    ws = G.Workspace(ds, grid, gp)
    stream = torch.cuda.current_stream()
    step = [0]

    def one_step():
        gp.step_index = step[0]
        G.push(ds, grid, gp, 1, workspace=ws, stats=False)
        step[0] += 1

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        one_step()
    barrier()
    clk = ClockSampler(local)
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    barrier()
    t0.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        one_step()
        ev[k][1].record(stream)
    t1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = t0.elapsed_time(t1)
    # steps that began with a sort run 3 more kernels; the push kernel's own
    # duration is taken from the steps without one
    first = args.warmup
    sorted_step = [args.sort_every > 0 and (first + k) % args.sort_every == 0
                   for k in range(args.steps)]
    step_ms = [a.elapsed_time(b) for a, b in ev]
    launch_ms = [t for t, srt in zip(step_ms, sorted_step) if not srt] or step_ms
    n_sorts = sum(sorted_step)
    tmax = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    ms = float(tmax.item())
    n = ds.n
    value = n * world * args.steps / (ms * 1e-3)
    stats = G.push(ds, grid, gp, 1, workspace=ws)

    # end to end through host buffers: per step, the state is copied in from
    # pinned host memory, pushed, and copied back out
    e2e = None
    if not args.no_e2e:
        host = [t.cpu().pin_memory() for t in ds.tensors()]
        dev = ds.tensors()
        h2d = sum(t.numel() * t.element_size() for t in host)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ke = max(3, args.steps // 5)
        e0.record(stream)
        for _ in range(ke):
            for d_, h_ in zip(dev, host):
                d_.copy_(h_, non_blocking=True)
            one_step()
            for d_, h_ in zip(dev, host):
                h_.copy_(d_, non_blocking=True)
        e1.record(stream)
        barrier()
        ems = e0.elapsed_time(e1)
        e2e = {"value": n * world * ke / (ems * 1e-3), "unit": METRIC,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d}

    fp64 = None
    if not args.no_fp64 and rank == 0:
        grid64 = G.Grid(fields, dtype="f64")
        d64 = G.State.from_numpy(st, precision="fp64")
        ws64 = G.Workspace(d64, grid64, gp)
        G.push(d64, grid64, gp, 1, workspace=ws64, stats=False)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        k64 = 3
        a.record(stream)
        G.push(d64, grid64, gp, k64, workspace=ws64, stats=False)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b) / k64
        fp64 = {"value": n / (ms64 * 1e-3), "unit": METRIC, "ms_per_step": ms64,
                "mixed_speedup": (value / world) / (n / (ms64 * 1e-3))}
        del grid64, d64

    if rank == 0:
        pk, src = peaks()
        avg_launch = sum(launch_ms) / len(launch_ms)
        achieved = alg_bytes_per_launch(n) / (avg_launch * 1e-3) / 1e9
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": workload_config(n * world, world, args.sort_every, tile),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                             "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                             "traffic": None, "kernel": "k_push_sr<float,2,1,2>",
                             "alg_bytes_per_particle_step": 2 * STATE_B + FIELD_B / n,
                             "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"},
                "e2e": e2e,
                "gpu_launches": args.steps + 3 * n_sorts,
                "sort": {"every": args.sort_every, "sorts_in_timed_region": n_sorts,
                         "ms_step_with_sort": (sum(t for t, q in zip(step_ms, sorted_step) if q)
                                               / max(1, n_sorts)),
                         "ms_push_kernel": sum(launch_ms) / len(launch_ms)},
                "clocks": clocks,
                "branch_mix": {"boris": stats["n_boris"], "gca": stats["n_gca"],
                               "mean_iter": stats["sum_iter"] / max(1, stats["n_gca"]),
                               "max_iter": stats["max_iter"], "nonconv": stats["n_nonconv"],
                               "gcafail": stats["n_gcafail"]},
                "fp64": fp64}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(fields, st, p)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
