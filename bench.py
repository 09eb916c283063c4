"""Throughput of the coupled guiding-center / Boris push on one GB300.

Default workload (the graded one): the 2D reconnection-like field (double
Harris sheet with a GEM-style flux perturbation, 64 random-phase Fourier
modes, E = -v_in x B) on a 2048 x 1024 periodic grid with float32 fields and
precomputed float32 gradient grids, 2^24 Maxwell-Juttner positrons and
electrons (theta = 1), dt = 0.45, |q/m| with max Omega_C dt = 1e5: the
mixed-precision path (float32 arithmetic, float32-pair positions).  A step is
one pass of the whole push over all particles, state resident in HBM; the
particles are re-sorted by cell every 8 steps inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload reconnection2d|harris2d_fp64|sheet3d|sheet3d_literal|kerr_wald|
                              adjoint2d]

Under torchrun every rank pushes its own particles (weak scaling, no
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


def _gen_reconnection(n, seed):
    from paper_2007_14401_gb300 import inputs
    return inputs.reconnection_2d(nx=2048, ny=1024, n_particles=n, seed=seed)


def _gen_harris(n, seed):
    from paper_2007_14401_gb300 import inputs
    return inputs.harris_2d(n_per_species=max(1, n // 4), seed=seed - 1)


def _gen_kerr(n, seed):
    from paper_2007_14401_gb300 import inputs
    return inputs.kerr_wald(n_particles=n, seed=seed + 3)


def _gen_sheet3d(n, seed):
    from paper_2007_14401_gb300 import inputs
    return inputs.current_sheet_3d(n=256, n_particles=n, seed=seed + 1)


def _gen_sheet3d_literal(n, seed):
    # the literal |q/m| of "Omega_C dt up to 1e6" (every particle GCA)
    from paper_2007_14401_gb300 import inputs
    return inputs.current_sheet_3d(n=256, n_particles=n, seed=seed + 1, Q=2.1e6)


# Algorithmic bytes per particle-step (PiC mode): the state read and written
# once (mixed 2D: x as 2 FP32 pairs 16 B + u 12 B + dxp 8 B + flags 1 B;
# FP64 2D: 16 + 24 + 16 + 1; mixed 3D: 24 + 12 + 12 + 1) plus every field
# record read once per step (node records of 48 B: 2D FP32 with gradients;
# 2D FP64 without gradients; 32 B: 3D FP32 without gradients).
WORKLOADS = {
    "reconnection2d": dict(
        gen=_gen_reconnection, n=1 << 24, precision="mixed", grid="f32", sort_every=8,
        tile=(1, 1), state_b=37, field_b=2048 * 1024 * 48, fp64_b=(57, 2048 * 1024 * 96),
        desc="2D double Harris + GEM + 64 modes, 2048x1024 grid, {n} particles",
        prec="mixed: FP32 fields and arithmetic, FP32-pair positions",
        extra=dict(grid=[2048, 1024], dt=0.45, omega_c_dt_max=1e5, curvature=1,
                   grad_mode="grid", gca_tol=1e-7),
        # FMA-pipe busy fraction of this kernel in its ncu capture
        # (sm__pipe_fma_cycles_active, 2^21 particles; profiles/)
        fma_pipe=0.288,
        # DRAM bytes (read + write) of one push launch at 2^24 particles, from
        # an ncu capture of this kernel (1 pass: dram__bytes_read.sum +
        # dram__bytes_write.sum = 722.01 MB + 560.56 MB)
        traffic_b=1282.57e6),
    "harris2d_fp64": dict(
        gen=_gen_harris, n=16384, precision="fp64", grid="f64", sort_every=0, tile=(1, 1),
        state_b=57, field_b=128 * 128 * 48, fp64_b=None,
        desc="2D Harris sheet 128x128, {n} particles (q/m = -1, -10, -1e2, -1e3)",
        prec="FP64 fields, state and arithmetic",
        extra=dict(grid=[128, 128], dt=1.0, curvature=1, grad_mode="dw", gca_tol=1e-7)),
    "kerr_wald": dict(
        gen=_gen_kerr, n=1 << 22, precision="ks", grid="f32", sort_every=0, tile=(1, 1),
        state_b=49, field_b=512 * 512 * 32, fp64_b=None,
        desc="Kerr-Schild a=0.9, Wald field + split monopole, 512x512 (log r, theta) grid, "
             "{n} electrons, |q/m| = 1e3",
        prec="FP32 field records, FP64 metric, state and arithmetic",
        extra=dict(grid=[512, 512], dt=0.02, spin=0.9),
        # FP64-issue bound: FP64 flops per particle-step as executed (2 DFMA
        # + DMUL + DADD, ncu thread-instruction counts of this kernel at 2^18
        # particles) against the FP64 FMA rate measured live (libgcb_peak.so);
        # the derived peak 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz = 1.2586
        # TFLOP/s is the fallback
        alu=dict(flops=1724.4, peak=1.2586, peak_kind="fp64",
                 peak_source="derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz "
                             "(ncu peak_sustained dfma 304 inst/clk)")),
    "sheet3d": dict(
        gen=_gen_sheet3d, n=1 << 26, precision="mixed", grid="f32", sort_every=8,
        tile=(1, 1, 1), state_b=49, field_b=256 ** 3 * 32, fp64_b=(73, 256 ** 3 * 48),
        desc="3D kinked Harris sheet 256^3, guide 0.3, {n} particles (70% MJ upstream, 30% "
             "power law in the sheet), |q/m| = 20",
        prec="mixed: FP32 fields and arithmetic, FP32-pair positions",
        extra=dict(grid=[256, 256, 256], dt=0.45, curvature=1, grad_mode="dw", gca_tol=1e-7),
        fma_pipe=0.329),
    "sheet3d_literal": dict(
        gen=_gen_sheet3d_literal, n=1 << 26, precision="mixed", grid="f32", sort_every=8,
        tile=(1, 1, 1), state_b=49, field_b=256 ** 3 * 32, fp64_b=(73, 256 ** 3 * 48),
        desc="3D kinked Harris sheet 256^3, guide 0.3, {n} particles (70% MJ upstream, 30% "
             "power law in the sheet), |q/m| = 2.1e6 (all GCA)",
        prec="mixed: FP32 fields and arithmetic, FP32-pair positions",
        extra=dict(grid=[256, 256, 256], dt=0.45, curvature=1, grad_mode="dw", gca_tol=1e-7)),
}


def _gen_adjoint(n, seed):
    from paper_2007_14401_gb300 import inputs
    return inputs.reconnection_2d_modes(nx=512, ny=256, n_particles=n, seed=seed)


# The adjoint workload: the reconnection field at 512 x 256 written as base +
# sum_m a_m pattern_m over its 64 modes; one step of the timed loop is the
# forward run of ADJ_STEPS pushes plus the reverse sweep for L = mean final
# kinetic energy, which yields dL/d(initial state) of every particle and
# dL/da_m.
ADJ_STEPS, ADJ_CKPT, ADJ_FIXED_ITERS = 256, 16, 6
ADJOINT = dict(gen=_gen_adjoint, n=1 << 20,
               desc="adjoint: 2D double Harris + GEM + 64 modes at 512x256, {n} particles, "
                    f"{ADJ_STEPS} steps, checkpoints every {ADJ_CKPT} (particles sorted by cell "
                    "at each), mixed FP32 forward + "
                    "FP32 adjoint, FP64 node accumulators; L = mean final kinetic energy, "
                    "gradients w.r.t. the 64 mode amplitudes and all initial states")


def omega_c_dt(fields, p, x, u, flags):
    """Omega_C dt = |q/m| |B(x)| dt / (c Gamma) of every particle (host
    diagnostic of the bench line, float64): |B| interpolated at x with the
    linear shape functions of the grid, Gamma from the full momentum."""
    B = np.sqrt(sum(np.asarray(b, dtype=np.float64) ** 2 for b in fields["B"]))
    shape = B.shape                       # (ny, nx) or (nz, ny, nx)
    nd = len(shape)
    dx = fields["dx"]
    c = p.get("c", 1.0)
    qm = np.abs(np.asarray(list(p["qm"]) + [0.0] * 4, dtype=np.float64))
    out = np.empty(x.shape[1])
    step = 1 << 21
    for a in range(0, x.shape[1], step):
        b = min(x.shape[1], a + step)
        s = [x[d, a:b] / dx[d] for d in range(nd)]
        i0 = [np.floor(v).astype(np.int64) for v in s]
        t = [v - i for v, i in zip(s, i0)]
        n_ax = list(reversed(shape))      # nodes along x, y, (z)
        acc = np.zeros(b - a)
        for o in range(1 << nd):
            w = np.ones(b - a)
            idx = []
            for d in range(nd):
                hi = (o >> d) & 1
                w *= t[d] if hi else 1.0 - t[d]
                idx.append((i0[d] + hi) % n_ax[d])
            acc += w * B[tuple(reversed(idx))]
        gam = np.sqrt(1.0 + np.sum(u[:, a:b].astype(np.float64) ** 2, axis=0) / c ** 2)
        out[a:b] = qm[(flags[a:b].astype(np.int64) >> 6) & 3] * acc * p["dt"] / (c * gam)
    return out


def coupling_report(G, multi, ds, grid, gp, ws, ks, snap, step_first, steps, fields, p):
    """Branch mix of the timed steps: the state at the first timed step is
    restored and the same steps are replayed (same step indices, hence the
    same sorts) one call each with its statistics, reduced over the ranks
    after every call; Omega_C dt of this rank's particles at the first timed
    step."""
    for t, s in zip(ds.tensors(), snap):
        t.copy_(s)
    tot = None
    for k in range(steps):
        gp.step_index = step_first + k
        s = G.push_ks(ds, grid, gp, 1) if ks else G.push(ds, grid, gp, 1, workspace=ws)
        s = multi.reduce_stats(s, device="cuda")
        if tot is None:
            tot = dict(s)
        else:
            for key, v in s.items():
                tot[key] = max(tot[key], v) if key == "max_iter" else tot[key] + v
    ps = tot["n_boris"] + tot["n_gca"]
    mix = {"timed_steps": steps, "particle_steps": ps, "boris": tot["n_boris"],
           "gca": tot["n_gca"], "boris_fraction": tot["n_boris"] / max(1, ps),
           "to_gca": tot["n_to_gca"], "to_boris": tot["n_to_boris"],
           "mean_iter": tot["sum_iter"] / max(1, tot["n_gca"]), "max_iter": tot["max_iter"],
           "nonconv": tot["n_nonconv"], "gcafail": tot["n_gcafail"],
           "nonfinite": tot["n_nonfinite"], "exited": tot["n_exited"]}
    if not ks:
        x = snap[0].double().cpu().numpy()
        if ds.x_lo is not None:
            x = x + snap[4].double().cpu().numpy()
        om = omega_c_dt(fields, p, x, snap[1].cpu().numpy(), snap[3].cpu().numpy())
        om = om[np.isfinite(om)]
        mix["omega_c_dt_first_step"] = {"min": float(om.min()), "median": float(np.median(om)),
                                        "max": float(om.max()),
                                        "particles": int(om.size)}
    return mix


def alu_peaks():
    """Fused multiply-add throughput of this GPU measured live (TFLOP/s):
    scalar FP32, packed FP32x2 and FP64 (libgcb_peak.so, CUDA events)."""
    import ctypes as C

    import torch
    from paper_2007_14401_gb300 import build as B
    lib = C.CDLL(B.build_peak())
    lib.gcb_peak_fma.argtypes = [C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double)]
    lib.gcb_peak_fma.restype = C.c_int
    out = {}
    for name, kind, iters in (("fp32", 0, 40000), ("fp32x2", 1, 20000), ("fp64", 2, 1500)):
        v = C.c_double(0.0)
        rc = lib.gcb_peak_fma(kind, iters, C.c_void_p(torch.cuda.current_stream().cuda_stream),
                              C.byref(v))
        out[name] = v.value if rc == 0 else None
    out["how"] = ("16 blocks x 256 threads per SM, 8 independent FMA chains a thread, "
                  "second of two launches timed with CUDA events")
    return out


def red_peaks():
    """Rate of scattered atomic additions of this GPU measured live (G ops/s,
    FP32 and FP64; libgcb_peak.so, CUDA events)."""
    import ctypes as C

    import torch
    from paper_2007_14401_gb300 import build as B
    lib = C.CDLL(B.build_peak())
    lib.gcb_peak_red.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double)]
    lib.gcb_peak_red.restype = C.c_int
    out = {}
    for name, dt in (("f32", 0), ("f64", 1)):
        for pat, suffix in ((0, ""), (1, "_scattered")):
            v = C.c_double(0.0)
            rc = lib.gcb_peak_red(dt, pat, 2000,
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(v))
            out[name + suffix] = v.value if rc == 0 else None
    out["how"] = ("8 blocks x 256 threads per SM, 2000 atomic additions a thread into an "
                  "L2-resident buffer, the 32 lanes of an instruction on consecutive elements "
                  "(the peak; *_scattered: on 32 different sectors); second of two launches "
                  "timed with CUDA events")
    return out


def pic_deposit(G, multi, ds, grid, p, sort_every, tile, ws, step, w, args, barrier, stream, n):
    """The PiC step with current deposition (gcb_push_deposit_sr): each step
    zeroes J, pushes with deposition and sums J over the ranks
    (multi.reduce_current); timed in blocks of K steps against the same
    number of plain pushes with the same sort schedule.  The deposition's
    cost is the difference; its atomic additions per second over that time
    are set against the measured scattered-atomic rate."""
    import torch
    prec = "fp64" if w["precision"] == "fp64" else "mixed"
    cur = G.Current(grid, (-1.0, 1.0), precision=prec)
    gp = G.make_params(p, sort_every=sort_every, sort_tile=tile)
    K = max(8, args.steps // 2)

    def block(dep):
        # start on a sort step so that both blocks sort alike
        k0 = step[0] + (-step[0]) % max(1, sort_every)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(K):
            gp.step_index = k0 + k
            if dep:
                cur.J.zero_()
                G.push(ds, grid, gp, 1, workspace=ws, stats=False, current=cur)
                multi.reduce_current(cur.J)
            else:
                G.push(ds, grid, gp, 1, workspace=ws, stats=False)
        e1.record(stream)
        barrier()
        step[0] = k0 + K
        return e0.elapsed_time(e1)

    block(True)   # warm-up of the deposition kernels
    ms_dep = block(True)
    ms_push = block(False)
    value, ms_dep_max, _ = multi.whole_job_rate(n, K, ms_dep, device="cuda")
    _, ms_push_max, _ = multi.whole_job_rate(n, K, ms_push, device="cuda")
    # counts of one more step (statistics on)
    cur.zero()
    gp.step_index = step[0]
    G.push(ds, grid, gp, 1, workspace=ws, stats=True, current=cur)
    step[0] += 1
    n_sorts = sum(1 for k in range(K) if sort_every > 0 and k % sort_every == 0)
    dep_ms = (ms_dep_max - ms_push_max) / K
    try:
        rp = red_peaks()
    except (OSError, RuntimeError) as exc:
        rp = {"error": str(exc)[:200]}
    f = "f64" if prec == "fp64" else "f32"
    atom = cur.n_atomics / n
    out = {"value": value, "unit": METRIC, "steps": K, "ms_per_step": ms_dep_max / K,
           "ms_per_step_push_only": ms_push_max / K, "deposit_ms_per_step": dep_ms,
           "vs_push_only": ms_push_max / ms_dep_max,
           "pieces_per_particle_step": cur.n_pieces / n, "atomics_per_particle_step": atom,
           "skipped": cur.n_skipped, "j_dtype": f,
           "gpu_launches": K + 6 * n_sorts,
           "method": "per step: J zeroed (torch), push with deposition (one kernel), J summed "
                     "over ranks; same sort schedule as the push-only block it is set against"}
    if dep_ms > 0 and rp.get(f):
        ach = atom * n / (dep_ms * 1e-3) / 1e9
        out["roofline"] = {"bound": "l2_atomics", "achieved": ach, "peak": rp[f],
                           "unit": "Gop/s", "frac": ach / rp[f],
                           "peak_scattered": rp.get(f + "_scattered"),
                           "note": "atomic additions of one step over the time the deposition "
                                   "adds to the push; peak measured live: " + rp["how"]}
    return out


def option_costs(G, multi, ds, grid, p, sort_every, tile, ws, step, args, barrier, stream):
    """ms per step of the push with each method option on (the exact drift
    frame, the evolved gyration phase, the mirror terms) against the plain
    push, each timed over the same number of steps from a sort step."""
    import torch
    K = max(8, args.steps // 4)
    out = {}
    for name, over in (("plain", {}), ("drift_frame_bt", {"drift_frame": 1}),
                       ("gyro_phase_evolve", {"gyro_phase": 1}), ("mirror_terms", {"mirror": 1})):
        gp = G.make_params(p, sort_every=sort_every, sort_tile=tile, **over)
        k0 = step[0] + (-step[0]) % max(1, sort_every)
        gp.step_index = k0
        G.push(ds, grid, gp, 1, workspace=ws, stats=False)          # warm-up
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(K):
            gp.step_index = k0 + 1 + k
            G.push(ds, grid, gp, 1, workspace=ws, stats=False)
        e1.record(stream)
        barrier()
        step[0] = k0 + 1 + K
        _, ms, _ = multi.whole_job_rate(ds.n, K, e0.elapsed_time(e1), device="cuda")
        out[name] = ms / K
    base = out["plain"]
    return {"ms_per_step": out, "vs_plain": {k: v / base for k, v in out.items()},
            "steps": K, "method": "each option timed over the same number of steps of the "
                                  "evolving state, from a sort step, with CUDA events"}


def graphed_rate(G, multi, ds, grid, p, sort_every, tile, ws, step, args, barrier, stream, n):
    """The same PiC steps captured in a CUDA graph (gcb.StepGraph) and
    replayed: the host issues one graph launch per K steps instead of K
    calls, which matters where a step is shorter than its issue."""
    import torch
    se = max(1, sort_every)
    K = max(8, (args.steps // 2 + se - 1) // se * se)
    gp = G.make_params(p, sort_every=sort_every, sort_tile=tile)
    gp.step_index = step[0] + (-step[0]) % se
    sg = G.StepGraph(ds, grid, gp, K, ws)
    sg.replay()                                   # warm-up
    barrier()
    reps = 2
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        sg.replay()
    e1.record(stream)
    barrier()
    step[0] = gp.step_index + K
    rate, ms, _ = multi.whole_job_rate(n, K * reps, e0.elapsed_time(e1), device="cuda")
    return {"value": rate, "unit": METRIC, "ms_per_step": ms / (K * reps),
            "steps_per_graph": K, "replays": reps,
            "method": "K pushes (with their sorts) captured once in a CUDA graph, the graph "
                      "replayed; each replay repeats the same step indices"}


def workload_config(w, n_total, ngpu, sort_every, sort_tile):
    cfg = {"workload": w["desc"].format(n=n_total), "particles": n_total,
           "particles_per_gpu": n_total // ngpu, "steps_per_call": 1,
           "sort_every": sort_every, "sort_tile": list(sort_tile),
           "l2": "inputs larger than L2 (particle state > 126 MB per GPU)"
                 if n_total // ngpu * w["state_b"] > 126e6 else "state fits L2"}
    cfg.update(w["extra"])
    return cfg


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


def _oracle_ks(fields, p):
    import oracle as O
    O.build()
    of = O.ks_grid_field(fields)
    kp = O.ks_params(p["a"], p["r_in"], p["r_out"])
    op = O.make_params(c=1.0, dt=p["dt"], f_rho=p["f_rho"], f_E=p["f_E"], qm=p["qm"],
                       max_iter=p["gca_max_iter"], tol=p["gca_tol"])
    dl = O.ks_cell_sizes(of, p["a"])
    return lambda st, n, threads: O.push_ks(st, of, kp, op, n, dl=dl, nthreads=threads)


def _oracle_push(fields, p):
    """A callable (state, n_steps, threads) running the FP64 oracle."""
    if "r_in" in p:
        return _oracle_ks(fields, p)
    O, of, op = _oracle_for(fields, p)
    return lambda st, n, threads: O.push_sr(st, of, op, n, nthreads=threads)


def _oracle_for(fields, p):
    import oracle as O
    O.build()
    of = O.grid_field(fields["E"], fields["B"], fields["dx"], dB=fields.get("dB"))
    op = O.make_params(dt=p["dt"], qm=p["qm"], f_rho=p["f_rho"], f_E=p["f_E"], dl=p["dl"],
                       curvature=p["curvature"], grad_mode=p["grad_mode"],
                       max_iter=p["gca_max_iter"], tol=p["gca_tol"])
    return O, of, op


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def cpu_baseline(fields, st, p, budget_s=15.0, n_sample=1 << 16):
    """The FP64 oracle (as it stands) on the host cores, on a bounded sample."""
    from paper_2007_14401_gb300 import inputs
    run = _oracle_push(fields, p)
    n_sample = min(n_sample, st["flags"].size)
    sub = inputs.subset(st, np.arange(n_sample))
    cores = _cores()
    t0 = time.perf_counter()
    run(sub, 1, cores)
    t1 = time.perf_counter() - t0
    steps = max(1, min(2000, int(budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    run(sub, steps, cores)
    dt = time.perf_counter() - t0
    return {"value": n_sample * steps / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{n_sample} particles x {steps} steps of the same workload, FP64 "
                      f"oracle (C, OpenMP over particles), {dt:.1f} s"}


def run_reference(args, rank, w):
    """The reference arm: the FP64 CPU oracle on a bounded sample per step."""
    if rank != 0:
        return 0
    fields, st, p = w["gen"](min(w["n"], 1 << 14), 1)
    run = _oracle_push(fields, p)
    cores = _cores()
    n = st["flags"].size
    for _ in range(args.warmup):
        run(st, 1, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run(st, 1, cores)
    dt = time.perf_counter() - t0
    v = n * args.steps / dt
    line = {"metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "precision": "FP64 oracle (plain C, OpenMP over particles, host cores)",
            "config": workload_config(w, w["n"] * args.gpus, args.gpus, w["sort_every"],
                                      w["tile"]),
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"{n} particles of the workload per step (bounded "
                                       f"sample) x {args.steps} steps, FP64 oracle"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def fused_launches(first, n_steps, fuse, sort_every):
    """Kernels of n_steps fused steps: one push per launch (at most fuse steps,
    none spanning a sort) plus the sort's 6 kernels at each sort step."""
    count, j = 0, 0
    while j < n_steps:
        g = first + j
        k = min(fuse, n_steps - j)
        if sort_every > 0:
            if g % sort_every == 0:
                count += 6
            k = min(k, sort_every - g % sort_every)
        count += 1
        j += k
    return count


def end_to_end(G, ds, grid, gp, ws, ks, step, args, barrier, stream, n, multi):
    """The metric through the public API with the state in pinned host
    memory: every step copies each particle's whole state host -> device,
    pushes it and copies it back.  The particles are streamed in chunks on
    three CUDA streams (copy in, push, copy out), so that one chunk's copies
    overlap another's push, as a caller streaming particles through the GPU
    would; a chunk's next copy in waits for its previous copy out."""
    import torch
    host_all = [t.cpu().pin_memory() for t in ds.tensors()]
    h2d = sum(t.numel() * t.element_size() for t in host_all)

    def rows(t, a_, b_):
        return [t[a_:b_]] if t.dim() == 1 else [t[r, a_:b_] for r in range(t.shape[0])]

    # at most --e2e-chunks chunks of at least 2^21 particles (smaller chunks
    # cost more in per-copy overhead than their overlap gains)
    C = max(1, min(args.e2e_chunks, n >> 21))
    edges = [((n * c // C) // 256) * 256 for c in range(C)] + [n]
    spans = [(a_, b_) for a_, b_ in zip(edges[:-1], edges[1:]) if b_ > a_]
    views = [ds.view(a_, b_) for a_, b_ in spans]
    pairs = [[(d_, h_) for t_d, t_h in zip(ds.tensors(), host_all)
              for d_, h_ in zip(rows(t_d, a_, b_), rows(t_h, a_, b_))] for a_, b_ in spans]
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in spans]
    ev_cmp = [torch.cuda.Event() for _ in spans]
    ev_out = [torch.cuda.Event() for _ in spans]
    kws = G.ks_workspace() if ks else None
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ke = max(3, args.steps // 5)
    e0.record(stream)
    for s_ in (s_in, s_cmp, s_out):
        s_.wait_stream(stream)
    for k in range(ke):
        gp.step_index = step[0]
        for c, v in enumerate(views):
            if k > 0:
                s_in.wait_event(ev_out[c])
            with torch.cuda.stream(s_in):
                for d_, h_ in pairs[c]:
                    d_.copy_(h_, non_blocking=True)
            ev_in[c].record(s_in)
            s_cmp.wait_event(ev_in[c])
            if ks:
                G.push_ks(v, grid, gp, 1, stream=s_cmp, workspace=kws, stats=False)
            else:
                G.push(v, grid, gp, 1, stream=s_cmp, workspace=ws, stats=False)
            ev_cmp[c].record(s_cmp)
            s_out.wait_event(ev_cmp[c])
            with torch.cuda.stream(s_out):
                for d_, h_ in pairs[c]:
                    h_.copy_(d_, non_blocking=True)
            ev_out[c].record(s_out)
        step[0] += 1
    for s_ in (s_in, s_cmp, s_out):
        stream.wait_stream(s_)
    e1.record(stream)
    barrier()
    rate, _, _ = multi.whole_job_rate(n, ke, e0.elapsed_time(e1), device="cuda")
    return {"value": rate, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
            "chunks": len(spans), "streams": "copy-in / push / copy-out"}


def end_to_end_host(G, ds, grid, gp, ws, ks, step, args, barrier, stream, n, multi):
    """The metric through the public API with the particle state left in
    pinned host memory: every step the push kernels read the state from host
    memory and write it back there across the host link (NVLink-C2C on a
    Grace host), with no staging copies; the grid and the workspace stay in
    device memory."""
    import torch
    host = G.State(ds.n, ds.ndim, ds.precision,
                   pos_mode="pair" if ds.x_lo is not None else "f64", device="pinned",
                   with_pid=ds.pid is not None)
    for h, d in zip(host.tensors(), ds.tensors()):
        h.copy_(d)
    torch.cuda.synchronize()
    nbytes = sum(t.numel() * t.element_size() for t in host.tensors())
    kws = G.ks_workspace() if ks else None

    def one():
        gp.step_index = step[0]
        if ks:
            G.push_ks(host, grid, gp, 1, workspace=kws, stats=False)
        else:
            G.push(host, grid, gp, 1, workspace=ws, stats=False)
        step[0] += 1

    one()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ke = max(3, args.steps // 5)
    e0.record(stream)
    for _ in range(ke):
        one()
    e1.record(stream)
    barrier()
    rate, _, _ = multi.whole_job_rate(n, ke, e0.elapsed_time(e1), device="cuda")
    del host
    return {"value": rate, "unit": METRIC, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "steps": ke,
            "method": "state in pinned host memory, read and written in place by the push "
                      "kernels over the host link (no staging copies)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gcb", choices=["gcb", "reference"])
    ap.add_argument("--workload", default="reconnection2d",
                    choices=sorted(WORKLOADS) + ["adjoint2d"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fused", action="store_true",
                    help="skip the test-particle (fused-step) measurement")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint / forward cost ratio of the default line")
    ap.add_argument("--no-deposit", action="store_true",
                    help="skip the PiC step with current deposition")
    ap.add_argument("--no-options", action="store_true",
                    help="skip the cost of the method options (exact frame, phase, mirror)")
    ap.add_argument("--no-graph", action="store_true",
                    help="skip the CUDA-graph replay of the steps")
    ap.add_argument("--e2e-chunks", type=int, default=8,
                    help="particle chunks streamed through the GPU in the end-to-end timing")
    ap.add_argument("--sort-every", type=int, default=None)
    ap.add_argument("--sort-tile", default=None, help="cells per sort tile, e.g. 2,2")
    ap.add_argument("--ks-kick", default="tetrad", choices=["tetrad", "global"],
                    help="kerr_wald: basis of the GREOM half kicks (local frame or global)")
    ap.add_argument("--particles", type=int, default=None,
                    help="particles per GPU (smaller cases for profiling only)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload == "adjoint2d":
        if args.impl == "reference":
            if int(os.environ.get("RANK", "0")) == 0:
                print(json.dumps({"impl": "reference", "unavailable":
                                  "the CPU oracle has no adjoint; its gradient reference is central "
                                  "differences of the forward oracle, run on samples in the tests"}),
                      flush=True)
            return 0
        return run_adjoint(args)
    w = WORKLOADS[args.workload]
    sort_every = w["sort_every"] if args.sort_every is None else args.sort_every
    tile = w["tile"] if args.sort_tile is None else tuple(int(v) for v in args.sort_tile.split(","))
    n_req = w["n"] if args.particles is None else args.particles

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, w)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2007_14401_gb300 import gcb as G
    from paper_2007_14401_gb300 import multi

    fields, st, p = w["gen"](n_req, multi.rank_seed(rank))
    ks = w["precision"] == "ks"
    if ks:
        grid = G.KsGrid(fields, p["a"], p["r_in"], p["r_out"], dtype=w["grid"],
                        kick_basis=G.KS_GLOBAL if args.ks_kick == "global" else G.KS_TETRAD)
        ds = G.State.from_numpy(st, precision="fp64")
    else:
        grid = G.Grid(fields, dtype=w["grid"])
        ds = G.State.from_numpy(st, precision=w["precision"], pos_mode="pair")
    gp = G.make_params(p, sort_every=sort_every, sort_tile=tile)
    ws = G.Workspace(ds, grid, gp) if not ks else None
    stream = torch.cuda.current_stream()
    step = [0]

    def push(n):
        if ks:
            return G.push_ks(ds, grid, gp, n, stats=False)
        return G.push(ds, grid, gp, n, workspace=ws, stats=False)

    def one_step():
        gp.step_index = step[0]
        push(1)
        step[0] += 1

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        one_step()
    barrier()
    # the state at the first timed step, for replaying the timed steps with
    # their statistics afterwards (the push is deterministic per particle)
    snap, step_first = [t.clone() for t in ds.tensors()], step[0]
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
    # steps that began with a sort run 6 more kernels; the push kernel's own
    # duration is taken from the steps without one
    first = args.warmup
    sorted_step = [sort_every > 0 and (first + k) % sort_every == 0 for k in range(args.steps)]
    step_ms = [a.elapsed_time(b) for a, b in ev]
    launch_ms = [t for t, srt in zip(step_ms, sorted_step) if not srt] or step_ms
    n_sorts = sum(sorted_step)
    n = ds.n
    # whole job: all ranks' particle-steps over the slowest rank's time
    value, ms, n_all = multi.whole_job_rate(n, args.steps, ms, device="cuda")
    mix = coupling_report(G, multi, ds, grid, gp, ws, ks, snap, step_first, args.steps, fields,
                          p)
    del snap

    # end to end through host buffers: per step, the state is copied in from
    # pinned host memory, pushed, and copied back out
    e2e = None
    if not args.no_e2e:
        streamed = end_to_end(G, ds, grid, gp, ws, ks, step, args, barrier, stream, n, multi)
        streamed["method"] = "state copied from pinned host memory to the device and back every step"
        e2e = end_to_end_host(G, ds, grid, gp, ws, ks, step, args, barrier, stream, n, multi)
        if streamed["value"] > e2e["value"]:
            e2e, other = streamed, e2e
        else:
            other = streamed
        e2e = dict(e2e, other_method=other)

    # the test-particle mode (reported beside the graded PiC mode): up to 8
    # steps per launch with the state on chip between them, sorting as above
    tpm = None
    if not ks and not args.no_fused:
        fuse = 8
        gpf = G.make_params(p, sort_every=sort_every, sort_tile=tile, fuse_steps=fuse)
        gpf.step_index = step[0]
        G.push(ds, grid, gpf, fuse, workspace=ws, stats=False)
        step[0] += fuse
        barrier()
        kf = max(2, args.steps // fuse)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        gpf.step_index = step[0]
        f0.record(stream)
        G.push(ds, grid, gpf, fuse * kf, workspace=ws, stats=False)
        f1.record(stream)
        barrier()
        step[0] += fuse * kf
        tp_rate, tp_ms, _ = multi.whole_job_rate(n, fuse * kf, f0.elapsed_time(f1), device="cuda")
        tpm = {"value": tp_rate, "unit": METRIC, "fuse_steps": fuse, "steps": fuse * kf,
               "ms_per_step": tp_ms / (fuse * kf), "vs_pic_mode": tp_rate / value,
               "gpu_launches": fused_launches(gpf.step_index, fuse * kf, fuse, sort_every),
               "note": "state kept on chip across the fused steps; bound by instruction "
                       "issue (the ALU side), not HBM"}

    # the PiC step: push with current deposition and the current summed over
    # the ranks (reported beside the graded push)
    pic = None
    if not ks and not args.no_deposit:
        pic = pic_deposit(G, multi, ds, grid, p, sort_every, tile, ws, step, w, args, barrier,
                          stream, n)

    # what the method options cost on this workload (flat pushes with
    # FP32-pair positions or FP64: where every option has kernels)
    opts = None
    if not ks and not args.no_options:
        opts = option_costs(G, multi, ds, grid, p, sort_every, tile, ws, step, args, barrier,
                            stream)

    graphed = None
    if not ks and not args.no_graph:
        graphed = graphed_rate(G, multi, ds, grid, p, sort_every, tile, ws, step, args,
                               barrier, stream, n)
        graphed["vs_eager"] = graphed["value"] / value

    fp64 = None
    if not args.no_fp64 and rank == 0 and w["fp64_b"] is not None:
        n64 = min(n, 1 << 22)
        from paper_2007_14401_gb300 import inputs
        st64 = inputs.subset(st, np.arange(n64)) if n64 < n else st
        grid64 = G.Grid(fields, dtype="f64")
        d64 = G.State.from_numpy(st64, precision="fp64")
        gp64 = G.make_params(p)
        ws64 = G.Workspace(d64, grid64, gp64)
        G.push(d64, grid64, gp64, 1, workspace=ws64, stats=False)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        k64 = 3
        a.record(stream)
        G.push(d64, grid64, gp64, k64, workspace=ws64, stats=False)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b) / k64
        v64 = n64 / (ms64 * 1e-3)
        fp64 = {"value": v64, "unit": METRIC, "ms_per_step": ms64, "particles": n64,
                "mixed_speedup": (value / world) / v64}
        del grid64, d64

    if rank == 0:
        pk, src = peaks()
        avg_launch = sum(launch_ms) / len(launch_ms)
        alg = 2 * w["state_b"] * n + w["field_b"]
        achieved = alg / (avg_launch * 1e-3) / 1e9
        if ks:
            kname = "k_push_ks<float>"
        elif w["precision"] == "fp64":
            kname = "k_push_sr<double,2,0,1>"
        else:
            kname = "k_push_sr<float,{},1,{}>".format(
                len(w["extra"]["grid"]), 2 if w["extra"]["grad_mode"] == "grid" else 1)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                    "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                    "frac_of_nominal_8000_gbs": achieved / 8000.0,
                    "traffic": (w["traffic_b"] if "traffic_b" in w and n == w["n"] else None),
                    "kernel": kname, "alg_bytes_per_particle_step": alg / n,
                    "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"}
        try:
            apk = alu_peaks()
        except (OSError, RuntimeError) as exc:
            apk = {"error": str(exc)[:200]}
        if "alu" in w:
            a_ = w["alu"]
            tf = a_["flops"] * n / (avg_launch * 1e-3) / 1e12
            live = apk.get(a_["peak_kind"])
            peak_v, peak_src = (live, "measured live: " + apk["how"]) if live else \
                (a_["peak"], a_["peak_source"])
            roofline = {"bound": "alu", "achieved": tf, "peak": peak_v, "unit": "TFLOP/s",
                        "frac": tf / peak_v, "traffic": None, "kernel": kname,
                        "fp64_flops_per_particle_step": a_["flops"],
                        "peak_source": peak_src, "derived_peak": a_["peak"],
                        "hbm": {"achieved_gbs": achieved, "frac": achieved / pk["hbm_gbs"]}}
        elif "fma_pipe" in w:
            roofline["alu"] = {"fma_pipe_busy_frac": w["fma_pipe"],
                               "source": "ncu sm__pipe_fma_cycles_active of this kernel "
                                         "(profiles/)",
                               "measured_fma_tflops": {k: apk.get(k) for k in
                                                       ("fp32", "fp32x2", "fp64")}}
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if w["precision"] == "mixed" else "f64", "data": "synthetic",
                "precision": w["prec"],
                "config": dict(workload_config(w, n_all, world, sort_every, tile),
                               **({"kick_basis": args.ks_kick} if ks else {})),
                "roofline": roofline,
                "e2e": e2e,
                "gpu_launches": args.steps + 6 * n_sorts,
                "sort": {"every": sort_every, "sorts_in_timed_region": n_sorts,
                         "ms_step_with_sort": (sum(t for t, q in zip(step_ms, sorted_step) if q)
                                               / max(1, n_sorts)),
                         "ms_push_kernel": avg_launch},
                "clocks": clocks,
                "branch_mix": mix,
                "fp64": fp64, "test_particle_mode": tpm, "pic_deposit": pic,
                "option_costs": opts, "cuda_graph": graphed}
        if not args.no_adjoint and args.workload == "reconnection2d":
            line["adjoint_vs_forward"] = adjoint_vs_forward(G)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(fields, st, p)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def adjoint_launches():
    """Kernels of one forward + reverse sweep.  Forward: a sort (6 kernels)
    at each checkpoint, ADJ_STEPS pushes, then the composed order (one
    permutation per later checkpoint) and the scatter back to the caller's
    order.  Sweep: the composed order again and the gather of the adjoint
    into it; per segment its recomputed pushes, its adjoint steps and the
    adjoint's scatter to the previous checkpoint's order; the mode
    projection."""
    nck = (ADJ_STEPS + ADJ_CKPT - 1) // ADJ_CKPT
    seg = [min(ADJ_CKPT, ADJ_STEPS - s * ADJ_CKPT) for s in range(nck)]
    forward = 6 * nck + ADJ_STEPS + (nck - 1) + 1
    sweep = (nck - 1) + 1 + sum((L - 1) + L + 1 for L in seg) + 1
    return forward + sweep


def adjoint_setup(G, n_req, seed, reduce=lambda g: g):
    """The adjoint workload on the current GPU: returns (n, lam, forward,
    backward, number of modes); forward() runs ADJ_STEPS pushes from the initial state storing
    the checkpoints, backward() the reverse sweep for L = mean final kinetic
    energy, returning dL/da_m (passed through ``reduce``)."""
    import torch
    base, pats, amps, st, p = ADJOINT["gen"](n_req, seed)
    grid = G.Grid(base, dtype="f32")
    base_rec = grid.rec.clone()
    pat_rec = torch.stack([G.Grid(q, dtype="f32").rec for q in pats]).contiguous()
    amps_d = torch.tensor(amps, dtype=torch.float64, device="cuda")
    G.grid_combine(grid, base_rec, pat_rec, amps_d)
    init = G.State.from_numpy(st, precision="mixed", pos_mode="pair")
    # checkpoints sorted by cell: the segments run on cell-ordered particles
    gp = G.make_params(p, gca_fixed_iters=ADJ_FIXED_ITERS, sort_every=ADJ_CKPT, sort_tile=(1, 1))
    n = init.n
    cur = init.clone()
    lam = torch.empty((7, n), dtype=torch.float32, device="cuda")
    aws = G.AdjointWorkspace(cur, grid, ADJ_STEPS, ADJ_CKPT, gp)

    def forward():
        # the forward pass stores the checkpoints the reverse sweep starts from
        for t_, s_ in zip(cur.tensors(), init.tensors()):
            t_.copy_(s_)
        G.push_ckpt(cur, grid, gp, ADJ_STEPS, aws)

    def backward():
        # dL/du_final for L = mean (Gamma - 1) c^2: u / (Gamma n)
        Gm = torch.sqrt(1.0 + (cur.u * cur.u).sum(0))
        lam.zero_()
        lam[2:5] = cur.u / (Gm * n)
        grad = G.adjoint(init, grid, gp, ADJ_STEPS, lam, ADJ_CKPT, workspace=aws)
        return reduce(G.grad_project(grid, grad, pat_rec))

    return n, lam, forward, backward, len(amps)


def adjoint_vs_forward(G, reps=3):
    """One GPU: the adjoint workload's forward (ADJ_STEPS pushes storing the
    checkpoints) and reverse sweep, each timed with CUDA events; medians of
    ``reps`` after one untimed pair."""
    import torch
    n, _, forward, backward, _ = adjoint_setup(G, ADJOINT["n"], 1)
    forward()
    backward()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    tf, tb = [], []
    for _ in range(reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        forward()
        e[1].record(stream)
        backward()
        e[2].record(stream)
        torch.cuda.synchronize()
        tf.append(e[0].elapsed_time(e[1]))
        tb.append(e[1].elapsed_time(e[2]))
    ms_f, ms_b = statistics.median(tf), statistics.median(tb)
    return {"workload": ADJOINT["desc"].format(n=n), "ms_forward": ms_f, "ms_reverse": ms_b,
            "reverse_over_forward": ms_b / ms_f, "reps": reps,
            "note": "forward = the push steps storing the checkpoints; reverse = recomputed "
                    "segments + the adjoint kernel per step + the mode projection"}


def run_adjoint(args):
    """Forward ADJ_STEPS pushes + reverse sweep on one GPU (replicas only under
    torchrun: each rank differentiates its own particles, and the 64 mode
    gradients would be summed once after the sweep)."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(local)
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2007_14401_gb300 import gcb as G
    from paper_2007_14401_gb300 import multi
    n_req = ADJOINT["n"] if args.particles is None else args.particles
    # the amplitudes are shared by all ranks: their gradients are summed
    n, lam, forward, backward, n_modes = adjoint_setup(G, n_req, multi.rank_seed(rank),
                                                       multi.sum_over_ranks)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup if args.steps > 1 else 1):
        forward()
        backward()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    k = max(1, args.steps)
    ef = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(k)]
    eb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(k)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(k):
        ef[i][0].record(stream)
        forward()
        ef[i][1].record(stream)
        eb[i][0].record(stream)
        ga = backward()
        eb[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms_f = statistics.median(a.elapsed_time(b) for a, b in ef)
    ms_b = statistics.median(a.elapsed_time(b) for a, b in eb)
    value, ms, _ = multi.whole_job_rate(n, ADJ_STEPS * k, t0.elapsed_time(t1), device="cuda")
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
                "steps": k, "warmup": args.warmup, "ms_per_step": ms / k,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": ADJOINT["desc"].format(n=n), "particles": n,
                           "push_steps_per_step": ADJ_STEPS, "ckpt_every": ADJ_CKPT,
                           "gca_fixed_iters": ADJ_FIXED_ITERS, "grid": [512, 256],
                           "modes": n_modes,
                           "l2": "particle state 39 MB fits L2; checkpoints 620 MB do not"},
                "adjoint": {"ms_forward": ms_f, "ms_reverse": ms_b,
                            "reverse_over_forward": ms_b / ms_f,
                            # a few chaotic trajectories overflow FP32 over
                            # 256 steps: count them rather than print a NaN
                            "lam0_nonfinite_particles": int((~torch.isfinite(lam).all(0)).sum()),
                            "dL_da_finite_modes": int(torch.isfinite(ga).sum()),
                            "dL_da_median_abs": float(ga[torch.isfinite(ga)].abs().median())
                            if bool(torch.isfinite(ga).any()) else None},
                "gpu_launches": k * adjoint_launches(), "clocks": clocks, "e2e": None}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
