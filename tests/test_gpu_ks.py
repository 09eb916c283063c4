"""Parity of the covariant (Kerr-Schild) CUDA path with the FP64 oracle.

FP64 records: one step from identical states reproduces the oracle's flags
bit-exactly where the switch margin exceeds 1e-12 and its state to a relative
1e-12 (fixed implicit-midpoint iteration count on both sides).  FP32 records
(FP32 field interpolation, FP64 everything else): within FP32 rounding.
Both bases of the GREOM half kicks (local frame, global coordinates) are
checked against the oracle's own kick in that basis, and against each other.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_14401_gb300 import inputs
from tests.helpers import copy_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14401_gb300 import gcb
    return gcb


@pytest.fixture(scope="module")
def wald():
    return inputs.kerr_wald(nr=96, nth=80, n_particles=3000, seed=41)


def oracle_setup(fields, p, **over):
    q = dict(p, **over)
    of = O.ks_grid_field(fields)
    kp = O.ks_params(q["a"], q["r_in"], q["r_out"], q.get("kick_basis", 0))
    op = O.make_params(c=1.0, dt=q["dt"], f_rho=q["f_rho"], f_E=q["f_E"], qm=q["qm"],
                       mu_mode=q.get("mu_mode", 0), force=q.get("force", 0),
                       max_iter=q.get("gca_max_iter", 16), fixed_iters=q.get("gca_fixed_iters", 0),
                       tol=q.get("gca_tol", 1e-7))
    return of, kp, op, O.ks_cell_sizes(of, q["a"])


def run_both(G, fields, st, p, n_steps=1, dtype="f64", **over):
    q = dict(p, **over)
    grid = G.KsGrid(fields, q["a"], q["r_in"], q["r_out"], dtype=dtype,
                    kick_basis=q.get("kick_basis", 0))
    ds = G.State.from_numpy(st, precision="fp64")
    gs = G.push_ks(ds, grid, G.make_params(q), n_steps)
    got = ds.to_numpy()
    ref = copy_state(st)
    of, kp, op, dl = oracle_setup(fields, p, **over)
    os_ = O.push_ks(ref, of, kp, op, n_steps, dl=dl)
    return got, ref, gs, os_, grid, dl


def margins(fields, st, p, **over):
    of, kp, op, dl = oracle_setup(fields, p, **over)
    m = np.empty(st["flags"].size)
    for i in range(m.size):
        _, _, _, det = O.ks_step_one(of, kp, op, st["x"][:, i], st["u"][:, i],
                                     int(st["flags"][i]), dl)
        m[i] = det.margin
    return m


def test_cell_sizes_match(G, wald):
    fields, st, p = wald
    grid = G.KsGrid(fields, p["a"], p["r_in"], p["r_out"], dtype="f64")
    dl_gpu = grid.dl.cpu().numpy().reshape(79, 95)
    dl_orc = O.ks_cell_sizes(O.ks_grid_field(fields), p["a"])
    assert np.allclose(dl_gpu, dl_orc, rtol=1e-13, atol=0)


@pytest.mark.parametrize("qm,force", [(-1e3, 0), (-3.0, 0), (-1e3, 1), (-1e3, 2), (-30.0, 0)])
def test_fp64_one_step(G, wald, qm, force):
    fields, st, p = wald
    over = dict(qm=(qm,), force=force, gca_fixed_iters=5)
    m = margins(fields, st, p, **over)
    got, ref, gs, os_, _, _ = run_both(G, fields, st, p, **over)
    robust = np.abs(m) > 1e-12
    assert not np.any((got["flags"] != ref["flags"]) & robust)
    same = got["flags"] == ref["flags"]
    assert same.mean() > 0.999
    dx = np.abs(got["x"] - ref["x"])[:, same]
    dx[2] = np.minimum(dx[2], 2 * np.pi - dx[2])
    assert np.all(dx <= 1e-12 * np.maximum(np.abs(ref["x"][:, same]), 1.0))
    un = np.linalg.norm(ref["u"][:, same], axis=0) + 1.0
    assert np.all(np.abs(got["u"] - ref["u"])[:, same] <= 1e-12 * un)
    for k in ("n_boris", "n_gca", "n_gcafail", "n_nonfinite", "n_exited", "sum_iter", "max_iter"):
        assert gs[k] == os_[k], k
    if force == 0 and qm == -30.0:
        assert gs["n_boris"] > 0 and gs["n_gca"] > 0


def test_fp64_tolerance_mode_and_ten_steps(G, wald):
    fields, st, p = wald
    got, ref, gs, os_, _, _ = run_both(G, fields, st, p, n_steps=10, qm=(-30.0,))
    same = (got["flags"] == ref["flags"])
    assert same.mean() > 0.99
    d = np.abs(got["x"] - ref["x"])[:, same]
    d[2] = np.minimum(d[2], 2 * np.pi - d[2])
    assert np.median(d) < 1e-12 and np.max(d[0]) < 1e-6
    assert abs(gs["n_gca"] - os_["n_gca"]) <= 0.01 * max(1, os_["n_gca"])


def test_fp32_records_close_to_oracle(G, wald):
    fields, st, p = wald
    got, ref, gs, os_, _, _ = run_both(G, fields, st, p, dtype="f32", qm=(-1e3,),
                                       gca_fixed_iters=5)
    same = got["flags"] == ref["flags"]
    assert same.mean() > 0.995
    rel = np.abs(got["x"][0] - ref["x"][0]) / ref["x"][0]
    assert np.max(rel[same]) < 1e-6
    un = np.linalg.norm(ref["u"], axis=0) + 1.0
    assert np.max((np.abs(got["u"] - ref["u"]) / un)[:, same]) < 1e-4


def test_exits_and_frozen(G, wald):
    fields, st, p = wald
    st = copy_state(st)
    st["x"][0, :5] = p["r_in"] * 1.0001           # at the inner edge, falling in
    st["u"][0, :5] = -5.0
    st["u"][1, 7] = np.nan
    got, ref, gs, os_, _, _ = run_both(G, fields, st, p, n_steps=3, qm=(-3.0,),
                                       gca_fixed_iters=5)
    assert np.array_equal(got["flags"] & (G.FLAG_EXITED | G.FLAG_NONFINITE),
                          ref["flags"] & (O.FLAG_EXITED | O.FLAG_NONFINITE))
    assert np.all(got["flags"][:5] & G.FLAG_EXITED)
    assert gs["n_nonfinite"] == os_["n_nonfinite"] and gs["n_exited"] == os_["n_exited"]
    # the non-finite particle is not advanced in any of the 3 steps; the five
    # falling in leave at the first step and are frozen for the other two
    assert os_["n_nonfinite"] == 3 and os_["n_exited"] >= 10


@pytest.mark.parametrize("force", [1, 0])
def test_global_basis_one_step(G, wald, force):
    """GREOM half kicks in the global coordinate basis: flags and states as the
    oracle's global-basis kick, to the tolerance of the tetrad path."""
    fields, st, p = wald
    over = dict(qm=(-30.0,), force=force, gca_fixed_iters=5, kick_basis=G.KS_GLOBAL)
    m = margins(fields, st, p, **over)
    got, ref, gs, os_, _, _ = run_both(G, fields, st, p, **over)
    robust = np.abs(m) > 1e-12
    assert not np.any((got["flags"] != ref["flags"]) & robust)
    same = got["flags"] == ref["flags"]
    assert same.mean() > 0.999
    dx = np.abs(got["x"] - ref["x"])[:, same]
    dx[2] = np.minimum(dx[2], 2 * np.pi - dx[2])
    assert np.all(dx <= 1e-12 * np.maximum(np.abs(ref["x"][:, same]), 1.0))
    un = np.linalg.norm(ref["u"][:, same], axis=0) + 1.0
    assert np.all(np.abs(got["u"] - ref["u"])[:, same] <= 1e-12 * un)
    for k in ("n_boris", "n_gca", "n_gcafail", "n_nonfinite", "n_exited", "sum_iter", "max_iter"):
        assert gs[k] == os_[k], k
    assert gs["n_boris"] > 0


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_global_basis_equals_tetrad_on_gpu(G, wald, dtype):
    """The two bases compute one kick (det L = 1/sqrt(gamma)): ten steps of
    the CUDA path in each agree to rounding for every particle whose branch
    sequence is the same in both."""
    fields, st, p = wald
    out = []
    for basis in (G.KS_TETRAD, G.KS_GLOBAL):
        q = dict(p, qm=(-30.0,), gca_fixed_iters=5)
        grid = G.KsGrid(fields, q["a"], q["r_in"], q["r_out"], dtype=dtype, kick_basis=basis)
        ds = G.State.from_numpy(st, precision="fp64")
        stats = G.push_ks(ds, grid, G.make_params(q), 10)
        out.append((ds.to_numpy(), stats))
    (a, sa), (b, sb) = out
    same = a["flags"] == b["flags"]
    assert same.mean() > 0.999 and sa["n_boris"] > 0
    dx = np.abs(a["x"] - b["x"])[:, same]
    dx[2] = np.minimum(dx[2], 2 * np.pi - dx[2])
    dx /= np.maximum(np.abs(a["x"][:, same]), 1.0)
    assert np.median(dx) < 1e-13 and np.max(dx) < 1e-9
    un = np.linalg.norm(a["u"][:, same], axis=0) + 1.0
    du = np.abs(a["u"] - b["u"])[:, same] / un
    assert np.median(du) < 1e-13 and np.max(du) < 1e-9


def test_unknown_kick_basis_is_refused(G, wald):
    fields, st, p = wald
    with pytest.raises(RuntimeError, match="kick_basis"):
        G.KsGrid(fields, p["a"], p["r_in"], p["r_out"], kick_basis=3)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_ambient_region_on_gpu(G, dtype):
    """The ambient-region test of Sec. 4.2 through the CUDA path: electrons
    at rest at r = 5.5 r_g on the equator of the Wald field with
    Omega_C0 = 10, 1e2, 1e3, 1e4 c/r_g (one species each), 191 steps of
    2 pi / 60 to t = 20 r_g/c, f_rho = f_E = 1.  The branch of every step is
    the oracle's (Boris throughout for rho_C0 = 0.1 r_g, GRGCA throughout
    below), and so are the final positions (FP64 records: 1e-9 relative;
    FP32 records: FP32 interpolation)."""
    import math
    fields, _, p = inputs.kerr_wald(nr=256, nth=256, Qm=0.0, n_particles=1, seed=0)
    a = p["a"]
    x0 = np.array([5.5, math.pi / 2, 0.0])
    of = O.ks_grid_field(fields)
    D, B = O.ks_gather(of, x0[0], x0[1])
    m = O.ks_metric(a, x0[0], x0[1])
    Bn = math.sqrt(B @ m["gdn"] @ B)
    omegas = (10.0, 1e2, 1e3, 1e4)
    qm = tuple(-w / Bn for w in omegas)
    st = dict(x=np.repeat(x0[:, None], 4, axis=1), u=np.zeros((3, 4)), dxp=np.zeros((3, 4)),
              flags=(np.arange(4, dtype=np.uint8) << 6))
    q = dict(p, dt=2 * math.pi / 60, f_rho=1.0, f_E=1.0, qm=qm)
    grid = G.KsGrid(fields, a, p["r_in"], p["r_out"], dtype=dtype)
    ds = G.State.from_numpy(st, precision="fp64")
    gp = G.make_params(q)
    ref = copy_state(st)
    of_, kp, op, dl = oracle_setup(fields, q)
    Sg, So = [], []
    for _ in range(191):
        G.push_ks(ds, grid, gp, 1, stats=False)
        Sg.append(ds.flags.cpu().numpy() & G.FLAG_S)
        O.push_ks(ref, of_, kp, op, 1, dl=dl)
        So.append(ref["flags"] & O.FLAG_S)
    Sg, So = np.array(Sg), np.array(So)
    np.testing.assert_array_equal(Sg, So)
    assert Sg[:, 0].all() and not Sg[:, 1:].any()
    got = ds.to_numpy()
    tol = 1e-9 if dtype == "f64" else 1e-5
    np.testing.assert_allclose(got["x"], ref["x"], rtol=tol, atol=tol)
