"""The exact drift frame (gcb_params.drift_frame = GCB_FRAME_BT, Sec. 2.2) on
the GPU against the oracle's, through the C ABI.

Workload: the Harris sheet with a guide field and a uniform E_z (E.B = E_z B_z
!= 0 wherever B_z != 0), where b* and the exact v_E differ from the
simplified frame at first order in E.B.  FP64: one step from identical
states reproduces the oracle's flags where the switch margin exceeds 1e-12
and its state to a relative 1e-12 (fixed iteration count); the exact frame's
step differs from the simplified frame's by far more than that.  Mixed path:
within FP32 rounding of the oracle.  Where E.B = 0 (the reconnection field)
the two frames agree to rounding.  The paths that do not carry the option
refuse it.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_14401_gb300 import inputs
from tests.helpers import copy_state, oracle_field, oracle_params, switch_margins
from tests.test_gpu_parity import assert_fp64_parity, run_both

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14401_gb300 import gcb
    return gcb


def harris_eb(n_per=512, seed=4):
    """Harris sheet, guide field 0.3 and E_z = 0.08 (E.B = 0.024)."""
    return inputs.harris_2d(n_per_species=n_per, seed=seed, Bg=0.3, Ez=0.08)


@pytest.mark.parametrize("force", [0, 2])
def test_fp64_exact_frame_matches_oracle(G, force):
    fields, st, p = harris_eb()
    p = dict(p, gca_fixed_iters=6, force=force, drift_frame=O.FRAME_BT)
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    got, ref, gs, os_, _ = run_both(G, fields, st, p)
    frac = assert_fp64_parity(got, ref, m, (128.0, 128.0), (1.0, 1.0))
    assert frac > 0.999
    for k in ("n_boris", "n_gca", "n_gcafail", "sum_iter"):
        assert gs[k] == os_[k], (k, gs[k], os_[k])
    assert gs["n_gca"] > 100
    # the option changes the step well beyond the parity tolerance
    simple = copy_state(st)
    O.push_sr(simple, oracle_field(fields), oracle_params(dict(p, drift_frame=0)), 1)
    gca = (ref["flags"] & 1) == 0
    du = np.abs(simple["u"][:, gca] - ref["u"][:, gca]).max()
    assert du > 1e-6, du


def test_fp64_exact_frame_ten_steps(G):
    fields, st, p = harris_eb(n_per=256, seed=5)
    p = dict(p, gca_fixed_iters=6, drift_frame=O.FRAME_BT)
    got, ref, gs, os_, _ = run_both(G, fields, st, p, n_steps=10)
    same = got["flags"] == ref["flags"]
    assert same.mean() > 0.99
    d = np.abs(got["u"][:, same] - ref["u"][:, same]) / (np.linalg.norm(ref["u"][:, same], axis=0) + 1)
    assert np.median(d) < 1e-12 and np.quantile(d, 0.99) < 1e-9


def test_mixed_exact_frame_close_to_oracle(G):
    fields, st, p = harris_eb(seed=6)
    p = dict(p, gca_fixed_iters=6, drift_frame=O.FRAME_BT)
    got, ref, gs, os_, _ = run_both(G, fields, st, p, precision="mixed", pos_mode="pair")
    same = got["flags"] == ref["flags"]
    assert same.mean() > 0.98
    d = np.abs(got["u"][:, same] - ref["u"][:, same]) / (np.linalg.norm(ref["u"][:, same], axis=0) + 1)
    assert np.quantile(d, 0.99) < 1e-4
    assert gs["n_gca"] > 100


def test_frames_agree_where_E_dot_B_vanishes(G):
    """The reconnection field has E = -v_in x B, so E.B = 0: b* = b and the
    exact v_E equals c E x B/B^2, and the two frames' steps agree to
    rounding (FP64)."""
    fields, st, p = inputs.reconnection_2d(nx=64, ny=32, n_particles=2048, omega_dt_max=50.0,
                                           seed=7)
    p = dict(p, gca_fixed_iters=5)
    a, _, _, _, _ = run_both(G, fields, st, p, drift_frame=O.FRAME_BT)
    b, _, _, _, _ = run_both(G, fields, st, p, drift_frame=O.FRAME_SIMPLE)
    assert np.array_equal(a["flags"], b["flags"])
    d = np.abs(a["u"] - b["u"]) / (np.linalg.norm(b["u"], axis=0) + 1)
    assert d.max() < 1e-12


def test_paths_without_the_exact_frame_refuse_it(G):
    import torch
    fields, st, p = harris_eb(n_per=16)
    grid = G.Grid(fields, dtype="f32")
    ds = G.State.from_numpy(st, precision="mixed", pos_mode="f64")
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.push(ds, grid, G.make_params(p, drift_frame=1), 1)
    ds = G.State.from_numpy(st, precision="mixed", pos_mode="pair")
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.push(ds, grid, G.make_params(p, drift_frame=1, fuse_steps=4), 4)
    with pytest.raises(G.GcbError, match="EINVAL"):
        G.push(ds, grid, G.make_params(p, drift_frame=2), 1)
    lam = torch.zeros((7, ds.n), dtype=torch.float32, device="cuda")
    mfields, mst, mp = inputs.reconnection_2d(nx=32, ny=16, n_particles=64, seed=8)
    mgrid = G.Grid(mfields, dtype="f32")
    mds = G.State.from_numpy(mst, precision="mixed", pos_mode="pair")
    lam = torch.zeros((7, mds.n), dtype=torch.float32, device="cuda")
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.adjoint(mds, mgrid, G.make_params(mp, drift_frame=1, gca_fixed_iters=4), 2, lam)
