"""Adjoint of the flat-space push against central finite differences of the
FP64 oracle, through the C ABI and the autograd binding.

Observable: L = mean over particles of the final kinetic energy (Gamma - 1) c^2,
plus a random linear functional of the final x, u and dxp so that every
adjoint component is exercised.  Gradients with respect to every particle's
initial x, u, dxp and to the amplitudes a_m of the field modes (fields = base
+ sum_m a_m pattern_m) come from gcb_adjoint_sr; the reference is the oracle's
central difference with step h, compared only where the differences at h and
h/2 agree (the map is smooth at the scale of h there: no switch threshold,
cell face or wrap is crossed).  The adjoint holds each particle-step's branch
and iteration count fixed; the runs use a fixed iteration count so that the
oracle's map is the same function.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2007_14401_gb300 import inputs
from tests.helpers import copy_state, oracle_field, oracle_params

pytestmark = pytest.mark.gpu

CASE = dict(nx=64, ny=32, delta=2.0, n_modes=4, max_mode=2, n_particles=512, omega_dt_max=5.0,
            seed=3)
N_STEPS = 12
FIXED = dict(gca_fixed_iters=4)
H = 1e-6


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14401_gb300 import gcb
    return gcb


@pytest.fixture(scope="module")
def case():
    base, pats, amps, st0, params = inputs.reconnection_2d_modes(**CASE)
    rng = np.random.default_rng(11)
    n = st0["flags"].shape[0]
    w = dict(x=rng.normal(size=(2, n)) * 1e-3, u=rng.normal(size=(3, n)) * 1e-3,
             dxp=rng.normal(size=(2, n)) * 1e-1)
    return base, pats, amps, st0, params, w


def per_particle_L(st, st_ref, w, L):
    """L_i for every particle; positions enter as the periodic difference from
    st_ref (so that central differences across a wrap stay small)."""
    n = st["flags"].shape[0]
    G = np.sqrt(1.0 + (st["u"] ** 2).sum(0))
    dx = st["x"] - st_ref["x"]
    dx -= np.asarray(L)[:, None] * np.round(dx / np.asarray(L)[:, None])
    return ((G - 1.0) / n + (w["x"] * dx).sum(0) + (w["u"] * st["u"]).sum(0)
            + (w["dxp"] * st["dxp"]).sum(0))


def oracle_run(fields, st, params):
    s = copy_state(st)
    O.push_sr(s, oracle_field(fields), oracle_params(params, **FIXED), N_STEPS)
    return s


@pytest.fixture(scope="module")
def fd(case):
    """Oracle central differences at h and h/2: per-particle state gradients
    (7, n) and mode gradients (M,)."""
    base, pats, amps, st0, params, w = case
    fields = inputs.combine_fields(base, pats, amps)
    ref = oracle_run(fields, st0, params)
    Lbox = (CASE["nx"] * 1.0, CASE["ny"] * 1.0)
    n = st0["flags"].shape[0]
    out = {}
    for h in (H, H / 2):
        gs = np.zeros((7, n))
        for k in range(7):
            comp, row = (("x", k) if k < 2 else ("u", k - 2) if k < 5 else ("dxp", k - 5))
            scale = np.maximum(1.0, np.abs(st0[comp][row])) if comp == "u" else np.ones(n)
            Ls = []
            for sgn in (1, -1):
                s = copy_state(st0)
                s[comp][row] = s[comp][row] + sgn * h * scale
                Ls.append(per_particle_L(oracle_run(fields, s, params), ref, w, Lbox))
            gs[k] = (Ls[0] - Ls[1]) / (2 * h * scale)
        ga = np.zeros(len(amps))
        for m in range(len(amps)):
            Ls = []
            for sgn in (1, -1):
                a = amps.copy()
                a[m] += sgn * h
                Ls.append(per_particle_L(oracle_run(inputs.combine_fields(base, pats, a), st0,
                                                    params), ref, w, Lbox).sum())
            ga[m] = (Ls[0] - Ls[1]) / (2 * h)
        out[h] = (gs, ga)
    return out


# Rounding floor of a central difference: the per-particle observable is
# O(0.05) and its rounding, amplified along the run, stays near 1e-15
# absolute; divided by h = 1e-6 that is 1e-9 on the gradient.
FD_FLOOR = 1e-9


def smooth_mask(a, b, tol):
    scale = np.sqrt(np.mean(b ** 2)) + 1e-300
    return np.abs(a - b) <= tol * (np.abs(b) + scale) + FD_FLOOR


def rel_err(got, ref, scale):
    return np.maximum(np.abs(got - ref) - FD_FLOOR, 0.0) / (np.abs(ref) + scale)


def run_gpu(G, case, precision, pos_mode, gdt, ckpt_every=5, method="reverse", ckpt_fwd=True,
            sort=0, outputs=False):
    """Forward + adjoint through ModePush; returns (state grads (7, n), mode grads)."""
    import torch
    base, pats, amps, st0, params, w = case
    grid = G.Grid(inputs.combine_fields(base, pats, amps), dtype=gdt)
    base_rec = G.Grid(base, dtype=gdt).rec
    pat_rec = torch.stack([G.Grid(p, dtype=gdt).rec for p in pats]).contiguous()
    mdt = torch.float64 if precision == "fp64" else torch.float32
    dev = "cuda"
    x0 = torch.tensor(st0["x"], dtype=torch.float64, device=dev, requires_grad=True)
    u0 = torch.tensor(st0["u"], dtype=mdt, device=dev, requires_grad=True)
    d0 = torch.tensor(st0["dxp"], dtype=mdt, device=dev, requires_grad=True)
    a = torch.tensor(amps, dtype=torch.float64, device=dev, requires_grad=True)
    cfg = dict(grid=grid, base=base_rec, pat=pat_rec,
               params=G.make_params(params, sort_every=sort, sort_tile=(1, 1), **FIXED),
               n_steps=N_STEPS, ckpt_every=ckpt_every,
               flags=torch.tensor(st0["flags"], device=dev), precision=precision,
               pos_mode=pos_mode, method=method, ckpt_in_forward=ckpt_fwd)
    x, u, dxp = G.ModePush.apply(x0, u0, d0, a, cfg)
    n = u.shape[1]
    Gm = torch.sqrt(1.0 + (u.double() ** 2).sum(0))
    wt = {k: torch.tensor(v, device=dev) for k, v in w.items()}
    L = ((Gm - 1.0) / n).sum() + (wt["x"] * x).sum() + (wt["u"] * u.double()).sum() \
        + (wt["dxp"] * dxp.double()).sum()
    L.backward()
    gs = torch.cat([x0.grad, u0.grad.double(), d0.grad.double()]).cpu().numpy()
    if outputs:
        return gs, a.grad.cpu().numpy(), [t.detach().double().cpu().numpy() for t in (x, u, dxp)]
    return gs, a.grad.cpu().numpy()


def compare(got, fd, tol, min_frac):
    (g1, a1), (g2, a2) = fd[H], fd[H / 2]
    gs, ga = got
    for k in range(7):
        ok = smooth_mask(g1[k], g2[k], 1e-5)
        assert ok.mean() >= min_frac, (k, ok.mean())
        scale = np.sqrt(np.mean(g2[k][ok] ** 2)) + 1e-300
        err = rel_err(gs[k][ok], g2[k][ok], scale)
        assert np.quantile(err, 0.99) <= tol, (k, np.quantile(err, [0.5, 0.99]), err.max())
    okm = smooth_mask(a1, a2, 1e-5)
    assert okm.all(), (a1, a2)
    scale = np.sqrt(np.mean(a2 ** 2))
    err = rel_err(ga, a2, scale)
    assert err.max() <= tol, (ga, a2, err)


def test_branch_mix(G, case):
    """The case exercises both branches (GCA and Boris) during the run."""
    base, pats, amps, st0, params, w = case
    grid = G.Grid(inputs.combine_fields(base, pats, amps), dtype="f64")
    st = G.State.from_numpy(st0, precision="fp64", pos_mode="f64")
    s = G.push(st, grid, G.make_params(params, **FIXED), N_STEPS)
    tot = s["n_gca"] + s["n_boris"]
    assert 0.1 * tot < s["n_gca"] < 0.9 * tot, s


@pytest.mark.parametrize("method", ["reverse", "tangent"])
def test_adjoint_fp64_matches_oracle_fd(G, case, fd, method):
    compare(run_gpu(G, case, "fp64", "f64", "f64", method=method), fd, 1e-6, 0.97)


def test_reverse_and_tangent_agree(G, case):
    """Two constructions of the same transposed step (written-out reverse
    sweep; dual-number Jacobian columns): equal to FP64 rounding."""
    r = run_gpu(G, case, "fp64", "f64", "f64", method="reverse")
    t = run_gpu(G, case, "fp64", "f64", "f64", method="tangent")
    for k in range(7):
        sc = np.abs(t[0][k]).max()
        np.testing.assert_allclose(r[0][k], t[0][k], rtol=0, atol=1e-11 * sc)
    np.testing.assert_allclose(r[1], t[1], rtol=1e-10, atol=0)


def test_adjoint_checkpoint_interval_invariance(G, case):
    """Checkpoint spacing, and whether the checkpoints come from the forward
    (gcb_push_sr_ckpt) or from the adjoint's own forward pass, change only
    where states are recomputed: the gradients agree to the rounding of the
    FP64 atomic accumulation."""
    ref = run_gpu(G, case, "fp64", "f64", "f64", ckpt_every=N_STEPS)
    for ck, fwd in ((1, True), (5, True), (5, False), (N_STEPS, False)):
        got = run_gpu(G, case, "fp64", "f64", "f64", ckpt_every=ck, ckpt_fwd=fwd)
        np.testing.assert_allclose(got[0], ref[0], rtol=0, atol=1e-12 * np.abs(ref[0]).max())
        np.testing.assert_allclose(got[1], ref[1], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("precision,pos_mode,gdt", [("fp64", "f64", "f64"),
                                                     ("mixed", "pair", "f32")])
@pytest.mark.parametrize("ckpt_fwd", [True, False])
def test_sorted_checkpoints_change_nothing(G, case, precision, pos_mode, gdt, ckpt_fwd):
    """Sorting the particles by cell at every checkpoint only reorders the
    work: each particle's arithmetic is unchanged, so the forward outputs and
    the state adjoint (returned in the caller's order) are identical bit for
    bit, and the mode gradients equal to the rounding of the FP64 node
    accumulation."""
    ref = run_gpu(G, case, precision, pos_mode, gdt, ckpt_every=5, ckpt_fwd=ckpt_fwd,
                  outputs=True)
    got = run_gpu(G, case, precision, pos_mode, gdt, ckpt_every=5, ckpt_fwd=ckpt_fwd,
                  sort=5, outputs=True)
    for a, b in zip(got[2], ref[2]):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_allclose(got[1], ref[1], rtol=1e-9, atol=0)


def test_reverse_and_tangent_agree_mixed(G, case):
    """The FP32 constructions: written-out reverse sweep (shared-memory
    accumulation, FP32 fast division) against dual-number columns (direct
    FP64 atomics): equal to FP32 rounding of the different operation orders."""
    r = run_gpu(G, case, "mixed", "pair", "f32", method="reverse")
    t = run_gpu(G, case, "mixed", "pair", "f32", method="tangent")
    for k in range(7):
        sc = np.sqrt(np.mean(t[0][k] ** 2))
        err = np.abs(r[0][k] - t[0][k]) / (np.abs(t[0][k]) + sc)
        assert np.quantile(err, 0.99) <= 1e-3, (k, np.quantile(err, [0.5, 0.99]))
    sc = np.sqrt(np.mean(t[1] ** 2))
    assert np.all(np.abs(r[1] - t[1]) <= 1e-3 * (np.abs(t[1]) + sc)), (r[1], t[1])


@pytest.mark.parametrize("method", ["reverse", "tangent"])
def test_adjoint_mixed_close_to_fp64(G, case, fd, method):
    """FP32 forward + FP32 adjoint (FP32-pair positions, FP32 records) against
    the oracle's FP64 differences: FP32 tangent arithmetic."""
    compare(run_gpu(G, case, "mixed", "pair", "f32", method=method), fd, 2e-2, 0.97)


def test_grid_combine_and_project(G, case):
    import torch
    base, pats, amps, st0, params, w = case
    for gdt in ("f64", "f32"):
        grid = G.Grid(base, dtype=gdt)
        base_rec = grid.rec.clone()
        pat_rec = torch.stack([G.Grid(p, dtype=gdt).rec for p in pats]).contiguous()
        want = G.Grid(inputs.combine_fields(base, pats, amps), dtype=gdt).rec
        G.grid_combine(grid, base_rec, pat_rec, torch.tensor(amps))
        tol = 1e-15 if gdt == "f64" else 1e-6
        assert torch.allclose(grid.rec, want, rtol=0, atol=tol)
        gr = torch.randn(grid.rec.numel(), dtype=torch.float64, device="cuda")
        got = G.grad_project(grid, gr, pat_rec)
        ref = (pat_rec.double() * gr[None, :]).sum(1)
        assert torch.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_adjoint_rejects_unsupported(G, case):
    import torch
    base, pats, amps, st0, params, w = case
    grid = G.Grid(base, dtype="f64")
    st = G.State.from_numpy(st0, precision="fp64", pos_mode="f64")
    lam = torch.zeros((7, st.n), dtype=torch.float64, device="cuda")
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.adjoint(st, grid, G.make_params(params, gca_max_iter=40), 4, lam)
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.adjoint(st, grid, G.make_params(params, grad_mode=0), 4, lam)
