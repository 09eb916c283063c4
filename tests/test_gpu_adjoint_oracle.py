"""The adjoint of the CUDA library against the oracle's FP64 dual-number
gradient (oracle/gcb_oracle_grad.cpp), particle by particle.

Observable: L = sum over a set W of particles of (Gamma_final - 1) / n.  The
GPU's FP64 forward + reverse sweep (gcb_push_sr_ckpt + gcb_adjoint_sr through
gcb.ModePush) gives dL/du0 of every particle and dL/da_m of the field-mode
amplitudes; the oracle carries the derivatives of every particle's final
state with respect to (a, u0) through the same steps.  Both differentiate the
discrete map with each particle-step's branch and fixed-point iteration count
held, and the runs use a fixed iteration count, so they compute the same
derivative; they differ only by the rounding of two implementations.

The two implementations round differently at every step, and the
linearised dynamics amplifies those differences in the derivative as much as
in the trajectory.  So the comparison is conditioned on the orbit:
  - W: the particles whose trajectory the two sides compute alike (final
    state within 1e-11 relative);
  - Wc: those of W whose derivatives stay below 1e3 (moderately amplifying
    orbits).
On Wc, dL/du0 agrees particle by particle to 1e-10 relative, and dL/da_m
(the reverse sweep seeded on Wc only) agrees to 1e-10 relative.  On all of W
the 99th percentile stays within 1e-10 and the largest difference within
1e-6.  The fractions in W and Wc are asserted.

Cases: a small one (64 x 32, 4 modes, 512 particles, 12 steps, both the
reverse sweep and the dual-number columns of the CUDA library) and the
adjoint workload's 1024-particle subset (512 x 256, 64 modes, 256 steps,
6 fixed-point iterations, checkpoints every 16).
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_14401_gb300 import inputs
from tests.helpers import copy_state, oracle_params, periodic_diff

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14401_gb300 import gcb
    return gcb


def gpu_run(G, base, pats, amps, st0, params, n_steps, ckpt, fixed, mask, method="reverse"):
    """FP64 forward + adjoint; returns (dL/du0 (3, n), dL/da (M,), final state)."""
    import torch
    dev = "cuda"
    grid = G.Grid(inputs.combine_fields(base, pats, amps), dtype="f64")
    base_rec = G.Grid(base, dtype="f64").rec
    pat_rec = torch.stack([G.Grid(p, dtype="f64").rec for p in pats]).contiguous()
    x0 = torch.tensor(st0["x"], dtype=torch.float64, device=dev)
    u0 = torch.tensor(st0["u"], dtype=torch.float64, device=dev, requires_grad=True)
    d0 = torch.tensor(st0["dxp"], dtype=torch.float64, device=dev)
    a = torch.tensor(amps, dtype=torch.float64, device=dev, requires_grad=True)
    cfg = dict(grid=grid, base=base_rec, pat=pat_rec,
               params=G.make_params(params, gca_fixed_iters=fixed), n_steps=n_steps,
               ckpt_every=ckpt, flags=torch.tensor(st0["flags"], device=dev),
               precision="fp64", pos_mode="f64", method=method)
    x, u, dxp = G.ModePush.apply(x0, u0, d0, a, cfg)
    n = u.shape[1]
    Gm = torch.sqrt(1.0 + (u ** 2).sum(0))
    w = torch.tensor(mask, dtype=torch.float64, device=dev)
    L = (w * (Gm - 1.0) / n).sum()
    L.backward()
    fin = dict(x=x.detach().cpu().numpy(), u=u.detach().cpu().numpy(),
               dxp=dxp.detach().cpu().numpy())
    return u0.grad.cpu().numpy(), a.grad.cpu().numpy(), fin


def oracle_run(base, pats, amps, st0, params, n_steps, fixed):
    """Final state and d(Gamma_final)/d(a, u0) per particle (n, M + 3)."""
    s = copy_state(st0)
    jac = O.push_jac(s, base, pats, amps, oracle_params(params, gca_fixed_iters=fixed), n_steps)
    u = s["u"]
    Gf = np.sqrt(1.0 + (u * u).sum(0))
    dG = np.einsum("kn,nkj->nj", u / Gf, jac[:, 2:5, :])
    return s, dG


def same_trajectory(fin, ref, L, dG):
    dx = np.abs(periodic_diff(fin["x"], ref["x"], L)).max(0)
    du = (np.abs(fin["u"] - ref["u"]) / np.maximum(np.abs(ref["u"]), 1.0)).max(0)
    dd = np.abs(fin["dxp"] - ref["dxp"]).max(0)
    return (dx <= 1e-11 * max(L)) & (du <= 1e-11) & (dd <= 1e-11) & \
        np.all(np.isfinite(dG), axis=1)


def check(G, base, pats, amps, st0, params, n_steps, ckpt, fixed, L, min_frac, method):
    n = st0["flags"].size
    M = len(amps)
    ref, dG = oracle_run(base, pats, amps, st0, params, n_steps, fixed)
    # first pass: every particle seeded, to find the trajectories both agree on
    _, _, fin = gpu_run(G, base, pats, amps, st0, params, n_steps, ckpt, fixed, np.ones(n),
                        method)
    W = same_trajectory(fin, ref, L, dG)
    Wc = W & (np.abs(dG).max(1) < 1e3)
    assert W.mean() >= min_frac and Wc.mean() >= 0.5 * min_frac, (W.mean(), Wc.mean())
    gu, ga, _ = gpu_run(G, base, pats, amps, st0, params, n_steps, ckpt, fixed,
                        Wc.astype(float), method)
    gw, _, _ = gpu_run(G, base, pats, amps, st0, params, n_steps, ckpt, fixed,
                       W.astype(float), method)
    want_u = dG[:, M:].T / n                              # (3, n)
    want_a = (dG[Wc, :M]).sum(0) / n
    su = np.sqrt(np.mean(want_u[:, W] ** 2))
    err_c = np.abs(gu[:, Wc] - want_u[:, Wc]) / (np.abs(want_u[:, Wc]) + su)
    err_w = np.abs(gw[:, W] - want_u[:, W]) / (np.abs(want_u[:, W]) + su)
    rep = dict(W=float(W.mean()), Wc=float(Wc.mean()), du0_Wc_max=float(err_c.max()),
               du0_W_p99=float(np.quantile(err_w, 0.99)), du0_W_max=float(err_w.max()))
    assert err_c.max() <= TOL, rep
    assert np.quantile(err_w, 0.99) <= TOL and err_w.max() <= 1e-6, rep
    assert np.all(gu[:, ~Wc] == 0.0)
    sa = np.sqrt(np.mean(want_a ** 2))
    err_a = np.abs(ga - want_a) / (np.abs(want_a) + sa)
    rep["da_Wc_max"] = float(err_a.max())
    assert err_a.max() <= TOL, rep
    return rep


@pytest.mark.parametrize("method", ["reverse", "tangent"])
def test_adjoint_small_case_matches_dual_oracle(G, method):
    base, pats, amps, st0, p = inputs.reconnection_2d_modes(
        nx=64, ny=32, delta=2.0, n_modes=4, max_mode=2, n_particles=512, omega_dt_max=5.0,
        seed=3)
    rep = check(G, base, pats, amps, st0, p, 12, 5, 4, (64.0, 32.0), 0.95, method)
    print(dict(case=f"small ({method})", **rep))


def test_adjoint_workload_subset_matches_dual_oracle(G):
    """The adjoint workload (reconnection field at 512 x 256 as base + 64
    modes, 256 steps, 6 fixed-point iterations, checkpoints every 16) on a
    1024-particle subset of its 2^20 particles, in FP64."""
    base, pats, amps, st, p = inputs.reconnection_2d_modes(nx=512, ny=256, n_particles=1 << 20,
                                                          seed=1)
    st0 = inputs.subset(st, np.arange(0, 1 << 20, 1024))
    rep = check(G, base, pats, amps, st0, p, 256, 16, 6, (512.0, 256.0), 0.8, "reverse")
    print(dict(case="adjoint workload subset", **rep))
