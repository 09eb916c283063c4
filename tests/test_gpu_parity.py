"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

FP64 path: one step from identical states must reproduce the oracle's switch
flags bit-exactly wherever the criterion margin exceeds 1e-12, and its state
to a relative 1e-12 (positions and displacements relative to max(|x|, dx),
momenta relative to |u| + c).  Runs use a fixed fixed-point iteration count
so that both sides stop after the same number of iterations.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_14401_gb300 import inputs
from tests.helpers import (copy_state, oracle_field, oracle_params, periodic_diff,
                           switch_margins)

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14401_gb300 import gcb
    return gcb


def run_both(G, fields, st0, params, n_steps=1, precision="fp64", pos_mode="f64", **over):
    """Advance copies of st0 on the GPU and in the oracle; returns both."""
    gdt = "f64" if precision == "fp64" else "f32"
    grid = G.Grid(fields, dtype=gdt)
    dstate = G.State.from_numpy(st0, precision=precision, pos_mode=pos_mode)
    gp = G.make_params(params, **over)
    gstats = G.push(dstate, grid, gp, n_steps)
    got = dstate.to_numpy()
    ref = copy_state(st0)
    ostats = O.push_sr(ref, oracle_field(fields), oracle_params(params, **over), n_steps)
    return got, ref, gstats, ostats, grid


def assert_fp64_parity(got, ref, margins, L, dx, frozen_ok=True):
    fl_g, fl_o = got["flags"], ref["flags"]
    robust = np.abs(margins) > 1e-12
    bad = (fl_g != fl_o) & robust
    assert not bad.any(), f"flags differ at robust particles: {np.nonzero(bad)[0][:10]}"
    same = fl_g == fl_o
    xs = max(dx)
    dxs = periodic_diff(got["x"], ref["x"], L)[:, same]
    scale_x = np.maximum(np.abs(ref["x"][:, same]), xs)
    assert np.all(np.abs(dxs) <= RTOL * scale_x), np.max(np.abs(dxs) / scale_x)
    dd = np.abs(got["dxp"][:, same] - ref["dxp"][:, same])
    assert np.all(dd <= RTOL * scale_x), np.max(dd / scale_x)
    un = np.linalg.norm(ref["u"][:, same], axis=0) + 1.0
    du = np.abs(got["u"][:, same] - ref["u"][:, same])
    assert np.all(du <= RTOL * un), np.max(du / un)
    return same.mean()


def small_harris(n_per=512, seed=0):
    return inputs.harris_2d(n_per_species=n_per, seed=seed)


@pytest.mark.parametrize("force", [0, 1, 2])
def test_fp64_one_step_harris(G, force):
    fields, st, p = small_harris()
    p = dict(p, gca_fixed_iters=6, force=force)
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    got, ref, gs, os_, _ = run_both(G, fields, st, p)
    frac = assert_fp64_parity(got, ref, m, (128.0, 128.0), (1.0, 1.0))
    assert frac > 0.999
    for k in ("n_boris", "n_gca", "n_to_gca", "n_to_boris", "n_gcafail", "n_nonfinite",
              "sum_iter", "max_iter"):
        assert gs[k] == os_[k], (k, gs[k], os_[k])
    assert gs["sum_ekin"] == pytest.approx(os_["sum_ekin"], rel=1e-12)
    if force == 0:
        assert gs["n_gca"] > 100 and gs["n_boris"] > 100


@pytest.mark.parametrize("variant", ["nocurv", "uperp", "tol"])
def test_fp64_one_step_variants(G, variant):
    fields, st, p = small_harris(256, seed=3)
    over = dict(gca_fixed_iters=6)
    if variant == "nocurv":
        over["curvature"] = 0
    elif variant == "uperp":
        over["mu_mode"] = 1
    else:
        over = dict(gca_fixed_iters=0, gca_tol=1e-7)
    p = dict(p, **over)
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    got, ref, gs, os_, _ = run_both(G, fields, st, p)
    assert_fp64_parity(got, ref, m, (128.0, 128.0), (1.0, 1.0))
    assert gs["n_gca"] == os_["n_gca"] and gs["sum_iter"] == os_["sum_iter"]


def test_fp64_one_step_reconnection_grid_gradients(G):
    fields, st, p = inputs.reconnection_2d(nx=256, ny=128, n_particles=6000, seed=5)
    p = dict(p, gca_fixed_iters=5)
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    got, ref, gs, os_, _ = run_both(G, fields, st, p)
    assert_fp64_parity(got, ref, m, (256.0, 128.0), (1.0, 1.0))
    assert gs["n_gca"] > 1000


def test_fp64_one_step_3d(G):
    fields, st, p = inputs.current_sheet_3d(n=24, n_particles=3000, seed=7)
    p = dict(p, gca_fixed_iters=5)
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    got, ref, gs, os_, _ = run_both(G, fields, st, p)
    assert_fp64_parity(got, ref, m, (24.0,) * 3, (1.0,) * 3)
    assert gs["n_gca"] > 100 and gs["n_boris"] > 100


def test_fp64_multi_step_harris(G):
    """Ten steps: still within tolerance for particles whose flags agree."""
    fields, st, p = small_harris(256, seed=4)
    p = dict(p, gca_fixed_iters=6)
    got, ref, gs, os_, _ = run_both(G, fields, st, p, n_steps=10)
    same = got["flags"] == ref["flags"]
    assert same.mean() > 0.99
    d = periodic_diff(got["x"], ref["x"], (128.0, 128.0))[:, same]
    assert np.max(np.abs(d)) < 1e-9


def test_edge_cases(G):
    """Ragged tail, empty input, non-finite particles frozen, positions on the
    box edges, a B = 0 region (forced Boris there)."""
    fields, st, p = small_harris(8, seed=9)   # 32 particles: one ragged tile
    n = st["flags"].size
    st["x"][:, 0] = [0.0, 0.0]
    st["x"][:, 1] = [np.nextafter(128.0, 0), np.nextafter(128.0, 0)]
    st["u"][1, 2] = np.nan
    st["x"][0, 3] = np.inf
    fields["B"][0][60:68, :] = 0.0
    fields["B"][2][60:68, :] = 0.0
    st["x"][1, 4] = 64.5
    p = dict(p, gca_fixed_iters=6)
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    got, ref, gs, os_, _ = run_both(G, fields, st, p, n_steps=2)
    for i in (2, 3):
        assert got["flags"][i] & G.FLAG_NONFINITE and ref["flags"][i] & O.FLAG_NONFINITE
    assert gs["n_nonfinite"] == os_["n_nonfinite"] == 4
    ok = np.isfinite(ref["u"]).all(axis=0) & np.isfinite(ref["x"]).all(axis=0)
    assert np.all((got["x"][:, ok] >= 0) & (got["x"][:, ok] < 128.0))
    assert np.array_equal(got["flags"], ref["flags"])
    # empty input
    empty = {k: v[..., :0].copy() for k, v in st.items()}
    got0, ref0, gs0, _, _ = run_both(G, fields, empty, p)
    assert gs0["n_boris"] == 0 and got0["x"].shape == (2, 0)


@pytest.mark.parametrize("pos_mode", ["f64", "pair"])
def test_mixed_one_step_close_to_oracle(G, pos_mode):
    """Mixed path, one step: flags equal where the margin exceeds the FP32
    resolution of the criterion, states within FP32 rounding."""
    fields, st, p = inputs.reconnection_2d(nx=256, ny=128, n_particles=8192, seed=11)
    p = dict(p, gca_fixed_iters=5)
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    got, ref, gs, os_, _ = run_both(G, fields, st, p, precision="mixed", pos_mode=pos_mode)
    robust = np.abs(m) > 1e-4
    assert np.all(got["flags"][robust] == ref["flags"][robust])
    same = got["flags"] == ref["flags"]
    d = periodic_diff(got["x"], ref["x"], (256.0, 128.0))[:, same]
    assert np.max(np.abs(d)) < 1e-5
    un = np.linalg.norm(ref["u"][:, same], axis=0) + 1.0
    assert np.max(np.abs(got["u"][:, same] - ref["u"][:, same]) / un) < 1e-4


def test_invalid_arguments_rejected(G):
    fields, st, p = small_harris(8)
    grid = G.Grid(fields, dtype="f64")
    ds = G.State.from_numpy(st, precision="fp64")
    bad = G.make_params(p, dt=-1.0)
    with pytest.raises(G.GcbError, match="EINVAL"):
        G.push(ds, grid, bad, 1)
    with pytest.raises(G.GcbError, match="EUNSUPPORTED"):
        G.push(G.State.from_numpy(st, precision="mixed"), grid, G.make_params(p), 1)
