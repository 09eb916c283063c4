"""Parity at the benchmark workloads' full sizes, in the launch configuration
the benchmark times: the same generators, seeds, particle counts, precisions,
record types, fixed-point tolerance and per-cell sort cadence (every 8 steps,
starting with step 0), with particle ids carried so that sorted outputs can
be matched to their inputs.

The GPU advances every particle; the oracle recomputes a seeded sample one by
one from the same inputs (rounded on the host to the precision the device
state holds: FP32 momenta and displacements, FP32-pair positions):
  - step 0 (sort + push): per sampled particle, flags equal wherever the
    switch margin exceeds the precision of the criterion, states within the
    path's one-step tolerance (mixed: FP32 rounding; FP64: 1e-12 relative,
    loosened only where the two sides' fixed points stop one iteration apart);
  - 9 steps (two sorts): the error distribution over the sample (median and
    99th percentile), since FP32-vs-FP64 differences grow along chaotic orbits;
  - at any size: the ids stay a permutation of 0 .. n-1 and the per-branch
    counters account for every particle-step.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_14401_gb300 import inputs
from paper_2007_14401_gb300.multi import rank_seed
from tests.helpers import copy_state, oracle_field, oracle_params, periodic_diff, switch_margins

pytestmark = pytest.mark.gpu

SEED = rank_seed(0)     # the single-GPU benchmark's inputs
N_SAMPLE = 4096


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14401_gb300 import gcb
    return gcb


def round_like_device(st, precision):
    """The state as the device holds it after loading (host arithmetic only):
    FP32 momenta and displacements, positions as an FP32 pair hi + lo."""
    if precision == "fp64":
        return copy_state(st)
    out = copy_state(st)
    hi = st["x"].astype(np.float32)
    lo = (st["x"] - hi.astype(np.float64)).astype(np.float32)
    out["x"] = hi.astype(np.float64) + lo.astype(np.float64)
    out["u"] = st["u"].astype(np.float32).astype(np.float64)
    out["dxp"] = st["dxp"].astype(np.float32).astype(np.float64)
    return out


def take(st, idx):
    return {k: (v[..., idx].copy()) for k, v in st.items()}


def rows_by_pid(G, ds, pids):
    """Sampled particles of a device state, located by id after sorting."""
    import torch
    inv = torch.empty_like(ds.pid)
    inv[ds.pid] = torch.arange(ds.n, dtype=ds.pid.dtype, device=ds.pid.device)
    rows = inv[torch.as_tensor(pids, device=ds.pid.device)]
    x = ds.x_f64()[:, rows]
    out = dict(x=x.cpu().numpy(), u=ds.u[:, rows].double().cpu().numpy(),
               dxp=ds.dxp[:, rows].double().cpu().numpy(), flags=ds.flags[rows].cpu().numpy(),
               pid=ds.pid[rows].cpu().numpy())
    assert np.array_equal(out["pid"], pids)
    return out


def assert_permutation(ds):
    import torch
    seen = torch.zeros(ds.n, dtype=torch.int32, device=ds.pid.device)
    seen.index_add_(0, ds.pid, torch.ones_like(ds.pid, dtype=torch.int32))
    assert int(seen.min()) == 1 and int(seen.max()) == 1


def counted(stats, n, steps):
    return (stats["n_boris"] + stats["n_gca"] + stats["n_nonfinite"] + stats["n_exited"]
            == n * steps)


SWITCH_BITS = O.FLAG_S | O.FLAG_SPREV


def comparable(got, ref):
    """Particles whose switch bits agree and that neither side left
    unconverged (a fixed point that FP32 stops short of the tolerance while
    FP64 reaches it differs by the NONCONV bit alone; about 1 in 10^5 here)."""
    sw = (got["flags"] & SWITCH_BITS) == (ref["flags"] & SWITCH_BITS)
    nc = ((got["flags"] | ref["flags"]) & O.FLAG_NONCONV) != 0
    return sw & ~nc


# --------------------------------------------------------------------------
# flat workloads (mixed precision, sorted every 8 steps)
# --------------------------------------------------------------------------
FLAT = {
    "reconnection2d": dict(
        gen=lambda: inputs.reconnection_2d(nx=2048, ny=1024, n_particles=1 << 24, seed=SEED),
        L=(2048.0, 1024.0), tile=(1, 1)),
    "sheet3d": dict(
        gen=lambda: inputs.current_sheet_3d(n=256, n_particles=1 << 26, seed=SEED + 1),
        L=(256.0, 256.0, 256.0), tile=(1, 1, 1)),
}


@pytest.fixture(scope="module", params=sorted(FLAT))
def flat_run(request, G):
    import torch
    w = FLAT[request.param]
    fields, st, p = w["gen"]()
    n = st["flags"].size
    grid = G.Grid(fields, dtype="f32")
    ds = G.State.from_numpy(st, precision="mixed", pos_mode="pair", with_pid=True)
    gp = G.make_params(p, sort_every=8, sort_tile=w["tile"])
    ws = G.Workspace(ds, grid, gp)
    rng = np.random.default_rng(1234)
    pids = np.sort(rng.choice(n, size=N_SAMPLE, replace=False))
    st_dev = round_like_device(take(st, pids), "mixed")
    out = {}
    total = None
    for k in range(9):
        gp.step_index = k
        s = G.push(ds, grid, gp, 1, workspace=ws)
        total = s if total is None else {q: (total[q] + s[q] if q not in ("max_iter", "sum_ekin")
                                             else s[q]) for q in s}
        if k == 0:
            out["step1"] = rows_by_pid(G, ds, pids)
            assert_permutation(ds)
    out["step9"] = rows_by_pid(G, ds, pids)
    assert_permutation(ds)
    out["counted"] = counted(total, n, 9)
    del ds, ws, grid
    torch.cuda.empty_cache()
    return request.param, fields, p, pids, st_dev, out, w["L"]


def test_full_size_first_step_matches_oracle_per_particle(flat_run):
    name, fields, p, pids, st_dev, out, L = flat_run
    of, op = oracle_field(fields), oracle_params(p)
    m = switch_margins(of, op, st_dev)
    ref = copy_state(st_dev)
    O.push_sr(ref, of, op, 1)
    got = out["step1"]
    robust = np.abs(m) > 1e-4
    assert np.all((got["flags"] & SWITCH_BITS)[robust] == (ref["flags"] & SWITCH_BITS)[robust]), name
    same = comparable(got, ref)
    assert same.mean() > 0.999
    d = np.abs(periodic_diff(got["x"], ref["x"], L))[:, same]
    assert np.max(d) < 1e-5, (name, np.max(d))
    dd = np.abs(got["dxp"] - ref["dxp"])[:, same]
    assert np.max(dd) < 1e-5, (name, np.max(dd))
    un = np.linalg.norm(ref["u"][:, same], axis=0) + 1.0
    assert np.max(np.abs(got["u"] - ref["u"])[:, same] / un) < 1e-4, name


def test_full_size_nine_steps_statistics(flat_run):
    name, fields, p, pids, st_dev, out, L = flat_run
    assert out["counted"], "per-branch counters must cover every particle-step"
    ref = copy_state(st_dev)
    O.push_sr(ref, oracle_field(fields), oracle_params(p), 9)
    got = out["step9"]
    same = comparable(got, ref)
    assert same.mean() > 0.99, (name, same.mean())
    d = np.max(np.abs(periodic_diff(got["x"], ref["x"], L)), axis=0)[same] / max(L)
    assert np.median(d) < 1e-8 and np.quantile(d, 0.99) < 1e-6, \
        (name, np.median(d), np.quantile(d, 0.99))
    un = np.linalg.norm(ref["u"], axis=0) + 1.0
    du = np.max(np.abs(got["u"] - ref["u"]), axis=0)[same] / un[same]
    assert np.median(du) < 1e-5 and np.quantile(du, 0.99) < 1e-3, \
        (name, np.median(du), np.quantile(du, 0.99))


# --------------------------------------------------------------------------
# Harris FP64 (16 384 particles: compared in full)
# --------------------------------------------------------------------------
def test_full_size_harris_fp64(G):
    fields, st, p = inputs.harris_2d(n_per_species=16384 // 4, seed=SEED - 1)
    n = st["flags"].size
    assert n == 16384
    grid = G.Grid(fields, dtype="f64")
    ds = G.State.from_numpy(st, precision="fp64", with_pid=True)
    gp = G.make_params(p)
    stats = G.push(ds, grid, gp, 1)
    got = rows_by_pid(G, ds, np.arange(n))
    of, op = oracle_field(fields), oracle_params(p)
    m = switch_margins(of, op, st)
    ref = copy_state(st)
    O.push_sr(ref, of, op, 1)
    assert counted(stats, n, 1)
    robust = np.abs(m) > 1e-12
    assert np.all((got["flags"] & SWITCH_BITS)[robust] == (ref["flags"] & SWITCH_BITS)[robust])
    assert np.mean(got["flags"] == ref["flags"]) > 0.999
    same = comparable(got, ref)
    L = (128.0, 128.0)
    d = np.max(np.abs(periodic_diff(got["x"], ref["x"], L)), axis=0)[same]
    scale = np.max(np.maximum(np.abs(ref["x"][:, same]), 1.0), axis=0)
    # tolerance-stopped fixed points: both sides iterate the same FP64 map and
    # stop together except where the residual sits within rounding of the
    # tolerance, where they end one iterate (< tol) apart
    assert np.mean(d <= 1e-12 * scale) > 0.999
    assert np.max(d) < 10 * p["gca_tol"]
    un = np.linalg.norm(ref["u"][:, same], axis=0) + 1.0
    du = np.max(np.abs(got["u"] - ref["u"])[:, same], axis=0) / un
    assert np.mean(du <= 1e-12) > 0.999 and np.max(du) < 1e-5


# --------------------------------------------------------------------------
# Kerr-Schild (2^22 particles, FP32 records)
# --------------------------------------------------------------------------
def test_full_size_kerr(G):
    import torch
    fields, st, p = inputs.kerr_wald(n_particles=1 << 22, seed=SEED + 3)
    n = st["flags"].size
    grid = G.KsGrid(fields, p["a"], p["r_in"], p["r_out"], dtype="f32")
    ds = G.State.from_numpy(st, precision="fp64", with_pid=True)
    gp = G.make_params(p)
    stats = G.push_ks(ds, grid, gp, 1)
    rng = np.random.default_rng(99)
    pids = np.sort(rng.choice(n, size=N_SAMPLE // 2, replace=False))
    got = rows_by_pid(G, ds, pids)
    assert counted(stats, n, 1)
    del ds, grid
    torch.cuda.empty_cache()
    of = O.ks_grid_field(fields)
    kp = O.ks_params(p["a"], p["r_in"], p["r_out"])
    op = O.make_params(c=1.0, dt=p["dt"], f_rho=p["f_rho"], f_E=p["f_E"], qm=p["qm"],
                       tol=p.get("gca_tol", 1e-7), max_iter=p.get("gca_max_iter", 16))
    ref = take(st, pids)
    O.push_ks(ref, of, kp, op, 1, dl=O.ks_cell_sizes(of, p["a"]))
    same = got["flags"] == ref["flags"]
    assert same.mean() > 0.995
    rel = np.abs(got["x"][0] - ref["x"][0]) / ref["x"][0]
    assert np.max(rel[same]) < 1e-6
    dth = np.abs(got["x"][1] - ref["x"][1])
    assert np.max(dth[same]) < 1e-6
    un = np.linalg.norm(ref["u"], axis=0) + 1.0
    assert np.max((np.abs(got["u"] - ref["u"]) / un)[:, same]) < 1e-4
