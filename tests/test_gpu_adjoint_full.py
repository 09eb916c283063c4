"""The adjoint at the size of the adjoint benchmark, checked on a sample.

Launch configuration as timed: the 512 x 256 reconnection field with its 64
modes, 2^20 particles, 256 steps, checkpoints every 16 with the particles
sorted by cell at each, FP32 forward and FP32 adjoint with FP64 node
accumulators, L = mean final kinetic energy over all particles.  The
oracle cannot differentiate 2^20 particles, so the check runs
on a sample of 1024 of them (every 1024th), by central differences of the
FP64 oracle with h = 1e-6 (and h/2, to see where the map is smooth):

  - initial-momentum gradients: a particle's dL/du0 involves only its own
    trajectory, so N dL/du0_i from the full launch is compared with the
    oracle's d(Gamma_i - 1)/du0_i;
  - mode gradients: a second sweep at full size seeds the adjoint only on the
    sampled particles of the well-conditioned set W, so its dL_W/da_m is
    compared with the oracle's difference of L_W = mean over W of
    (Gamma_i - 1) for the first 8 modes.

Over 256 steps a few trajectories are chaotic (their derivatives reach 1e30
and more, and FP32 and FP64 trajectories part), so the comparison is
conditioned on W: particles whose oracle differences at h and h/2 agree in
every direction (smooth) and whose FP32 final momentum agrees with the
oracle's FP64 one to 1e-4.  The size of W is asserted, and the errors over
W are bounded at the median and the 99th percentile.

Set GCB_ERROR_REPORT=<file> to append the statistics as JSON lines.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2007_14401_gb300 import inputs
from tests.helpers import copy_state, oracle_field, oracle_params

pytestmark = pytest.mark.gpu

N = 1 << 20
N_STEPS = 256
CKPT = 16
FIXED = dict(gca_fixed_iters=6)
SAMPLE = np.arange(0, N, 1024)
N_MODES_FD = 8
H = 1e-6
FD_FLOOR = 1e-8


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14401_gb300 import gcb
    return gcb


def gamma_m1(u):
    return np.sqrt(1.0 + (u ** 2).sum(0)) - 1.0


@pytest.fixture(scope="module")
def problem():
    base, pats, amps, st, params = inputs.reconnection_2d_modes(nx=512, ny=256, n_particles=N,
                                                                seed=1)
    return base, pats, amps, st, params


def oracle_final(fields, st, params):
    s = copy_state(st)
    O.push_sr(s, oracle_field(fields), oracle_params(params, **FIXED), N_STEPS)
    return s


@pytest.fixture(scope="module")
def oracle_fd(problem):
    """FP64 oracle on the sample: final states and per-particle central
    differences of Gamma_i - 1 at h and h/2, for the 3 initial-momentum
    components (step h max(1, |u|)) and the first N_MODES_FD amplitudes."""
    base, pats, amps, st, params = problem
    sub = inputs.subset(st, SAMPLE)
    fields = inputs.combine_fields(base, pats, amps)
    ref = oracle_final(fields, sub, params)
    out = {}
    for h in (H, H / 2):
        gu = np.zeros((3, SAMPLE.size))
        for k in range(3):
            sc = np.maximum(1.0, np.abs(sub["u"][k]))
            e = []
            for sg in (1, -1):
                s = copy_state(sub)
                s["u"][k] = s["u"][k] + sg * h * sc
                e.append(gamma_m1(oracle_final(fields, s, params)["u"]))
            gu[k] = (e[0] - e[1]) / (2 * h * sc)
        ga = np.zeros((N_MODES_FD, SAMPLE.size))
        for m in range(N_MODES_FD):
            e = []
            for sg in (1, -1):
                a = amps.copy()
                a[m] += sg * h
                e.append(gamma_m1(oracle_final(inputs.combine_fields(base, pats, a), sub,
                                               params)["u"]))
            ga[m] = (e[0] - e[1]) / (2 * h)
        out[h] = (gu, ga)
    return ref, out


def run_full(G, problem, weights):
    """FP32 forward of all N particles, then the reverse sweep with
    lam_u = weights_i u_i / Gamma_i (weights: (N,) array or a scalar).
    Returns (final u (3, N) float64, lam0 (7, N) float64, dL/da_m (64,))."""
    import torch
    base, pats, amps, st, params = problem
    grid = G.Grid(base, dtype="f32")
    base_rec = grid.rec.clone()
    pat_rec = torch.stack([G.Grid(q, dtype="f32").rec for q in pats]).contiguous()
    G.grid_combine(grid, base_rec, pat_rec, torch.tensor(amps))
    init = G.State.from_numpy(st, precision="mixed", pos_mode="pair")
    # as the benchmark: particles sorted by cell at every checkpoint, the
    # forward storing the checkpoints (it returns the caller's order)
    gp = G.make_params(params, sort_every=CKPT, sort_tile=(1, 1), **FIXED)
    cur = init.clone()
    aws = G.AdjointWorkspace(cur, grid, N_STEPS, CKPT, gp)
    G.push_ckpt(cur, grid, gp, N_STEPS, aws)
    u = cur.u
    Gm = torch.sqrt(1.0 + (u * u).sum(0))
    w = torch.as_tensor(np.broadcast_to(weights, (N,)).astype(np.float32), device="cuda")
    lam = torch.zeros((7, N), dtype=torch.float32, device="cuda")
    fin = torch.isfinite(u).all(0)
    lam[2:5] = torch.where(fin, u / Gm * w, torch.zeros_like(u))
    grad = G.adjoint(init, grid, gp, N_STEPS, lam, CKPT, workspace=aws)
    ga = G.grad_project(grid, grad, pat_rec)
    torch.cuda.synchronize()
    return u.double().cpu().numpy(), lam.double().cpu().numpy(), ga.cpu().numpy()


def smooth(a, b, tol=1e-5):
    return np.abs(a - b) <= tol * (np.abs(b) + np.sqrt(np.mean(b ** 2))) + FD_FLOOR


def report(rec):
    path = os.environ.get("GCB_ERROR_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")


def test_adjoint_full_size_sample(G, problem, oracle_fd):
    ref, fd = oracle_fd
    (gu1, ga1), (gu2, ga2) = fd[H], fd[H / 2]
    u32, lam0, _ = run_full(G, problem, 1.0 / N)
    us = u32[:, SAMPLE]
    # the well-conditioned set W
    agree = np.all(np.abs(us - ref["u"]) <= 1e-4 * (np.abs(ref["u"]) + 1.0), axis=0)
    sm = np.all([smooth(gu1[k], gu2[k]) for k in range(3)], axis=0)
    sm &= np.all([smooth(ga1[m], ga2[m]) for m in range(N_MODES_FD)], axis=0)
    W = agree & sm
    rec = {"case": "adjoint 512x256, 2^20 particles, 256 steps, sample 1024",
           "frac_agree": float(agree.mean()), "frac_smooth": float(sm.mean()),
           "frac_W": float(W.mean())}
    # initial-momentum gradients over W: N dL/du0_i against d(Gamma_i - 1)/du0_i
    g = lam0[2:5][:, SAMPLE] * N
    errs = []
    for k in range(3):
        sc = np.sqrt(np.mean(gu2[k][W] ** 2))
        errs.append(np.abs(g[k][W] - gu2[k][W]) / (np.abs(gu2[k][W]) + sc))
    err = np.concatenate(errs)
    rec["du0_rel_err_median"], rec["du0_rel_err_p99"] = (float(np.median(err)),
                                                         float(np.quantile(err, 0.99)))
    # mode gradients of L_W through a second full-size sweep seeded on W only
    wts = np.zeros(N)
    wts[SAMPLE[W]] = 1.0 / W.sum()
    _, _, ga = run_full(G, problem, wts)
    fd_a = ga2[:, W].sum(1) / W.sum()
    sc = np.sqrt(np.mean(fd_a ** 2))
    erra = np.abs(ga[:N_MODES_FD] - fd_a) / (np.abs(fd_a) + sc)
    rec["da_rel_err_max"] = float(erra.max())
    rec["da_fd"] = fd_a.tolist()
    rec["da_adj"] = ga[:N_MODES_FD].tolist()
    report(rec)
    print(rec)
    # measured on a GB300 (6 fixed-point iterations): W 99.5 %, du0 1.8e-6
    # (median) / 1.2e-4 (p99), modes 1.9e-3 (max); the bounds leave about an
    # order of magnitude for the FP32 rounding differences between builds
    assert W.mean() >= 0.95, rec
    assert rec["du0_rel_err_median"] <= 1e-4 and rec["du0_rel_err_p99"] <= 1e-2, rec
    assert rec["da_rel_err_max"] <= 1e-2, rec
