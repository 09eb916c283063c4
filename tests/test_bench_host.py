"""Host-side logic of bench.py (no GPU): the reference arm's JSON line, its
rank handling, the adjoint workload's reference line, and the launch counts
the benchmark claims."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def run_bench(*args, env=None):
    e = dict(os.environ, **(env or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=e,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


@pytest.mark.parametrize("workload", ["harris2d_fp64", "kerr_wald"])
def test_reference_arm_line(workload):
    """One JSON line with the contract's keys: the oracle timed on the host
    cores, e2e equal to the value with no host-device bytes."""
    (line,) = run_bench("--impl", "reference", "--workload", workload, "--steps", "1",
                        "--warmup", "3")
    assert line["impl"] == "reference"
    assert line["metric"] == line["unit"] == "particle-steps/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    # the same config as the GPU arm's line (the workload, not a precision)
    w = bench.WORKLOADS[workload]
    assert line["config"] == json.loads(json.dumps(
        bench.workload_config(w, w["n"], 1, w["sort_every"], w["tile"])))
    assert "FP64 oracle" in line["precision"] and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "bounded sample" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    assert run_bench("--impl", "reference", "--workload", "harris2d_fp64", "--steps", "1",
                     env={"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_adjoint_reference_is_unavailable():
    (line,) = run_bench("--impl", "reference", "--workload", "adjoint2d")
    assert line["impl"] == "reference" and line["unavailable"]


@pytest.mark.parametrize("first,n_steps,fuse,sort_every,want", [
    (0, 16, 8, 8, 2 + 2 * 6),     # two launches of 8 steps, a sort before each
    (0, 16, 4, 8, 4 + 2 * 6),
    (3, 10, 8, 8, 2 + 6),         # steps 3-7, sort at 8, steps 8-12
    (0, 10, 8, 0, 2),             # no sorting: 8 + 2 steps
    (5, 1, 8, 8, 1),
])
def test_fused_launch_count(first, n_steps, fuse, sort_every, want):
    assert bench.fused_launches(first, n_steps, fuse, sort_every) == want


def test_adjoint_launch_count():
    """Forward: a sort at each of the 16 checkpoints (6 kernels each), 256
    pushes, 15 order compositions and the final scatter (368).  Sweep: 15
    compositions and the gather of the adjoint, then per segment 15
    recomputed pushes, 16 adjoint steps and one scatter, and the projection
    (529)."""
    assert (bench.ADJ_STEPS, bench.ADJ_CKPT) == (256, 16)
    assert bench.adjoint_launches() == 368 + 529


def test_omega_c_dt_closed_forms():
    """The bench line's Omega_C dt diagnostic: |q/m| |B| dt / (c Gamma) with
    |B| interpolated linearly between nodes (exact for a field linear in x,
    periodic wrap at the last cell), Gamma from the full momentum."""
    import numpy as np
    nx, ny = 8, 4
    X = np.tile(np.arange(nx, dtype=float), (ny, 1))
    Bz = 1.0 + 0.5 * X                     # |B| = 1 + x/2 on the nodes
    zero = np.zeros((ny, nx))
    fields = {"E": [zero, zero, zero], "B": [zero, zero, Bz], "dx": (1.0, 1.0)}
    p = {"qm": (-2.0, 3.0), "dt": 0.5, "c": 1.0}
    x = np.array([[0.0, 2.25, 6.5, 7.5], [0.1, 1.0, 3.9, 2.0]])
    u = np.array([[0.0, 1.0, 0.0, 0.0], [0.0, 0.0, 2.0, 0.0], [0.0, 0.0, 0.0, 0.0]])
    flags = np.array([0, 64, 0, 64], dtype=np.uint8)   # species 0, 1, 0, 1
    got = bench.omega_c_dt(fields, p, x, u, flags)
    Bx = np.array([1.0, 2.125, 4.25, 0.5 * (4.5 + 1.0)])     # last: wraps to node 0
    gam = np.sqrt(1 + np.array([0.0, 1.0, 4.0, 0.0]))
    want = np.array([2.0, 3.0, 2.0, 3.0]) * Bx * 0.5 / gam
    assert np.allclose(got, want, rtol=1e-14)
