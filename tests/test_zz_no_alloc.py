"""gcb_push_sr_noalloc: the push for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (a host callback or plugin hook that
forbids it, a device whose memory belongs to a pool they do not control, a
loop that must not allocate after start-up).  For them the library keeps its
scratch in a fixed device array and this entry point takes no workspace.
These tests call it through the C ABI and check it against gcb_push_sr with a
caller-provided workspace, twice in a row (the array keeps the previous
call's contents, so the second call checks that it is cleared where it must
be).  The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2007_14401_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-12   # the FP64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14401_gb300 import build
    build.build()
    from paper_2007_14401_gb300 import gcb
    return gcb


def noalloc_push(G, ds, grid, gp, n_steps):
    import torch
    st = G.GcbStats()
    rc = G.lib().gcb_push_sr_noalloc(C.byref(ds.s), C.byref(grid.s), C.byref(gp), n_steps,
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                     C.byref(st))
    return rc, {k: getattr(st, k) for k, _ in G.GcbStats._fields_}


def by_pid(out):
    if "pid" not in out:
        return out
    o = np.argsort(out["pid"])
    return {k: v[..., o] for k, v in out.items()}


def assert_same(a, b, stats_a, stats_b):
    assert np.array_equal(a["flags"], b["flags"])
    for k in ("x", "u", "dxp"):
        scale = np.maximum(np.abs(b[k]), 1.0)
        assert np.all(np.abs(a[k] - b[k]) <= RTOL * scale), k
    for k in ("n_boris", "n_gca", "n_to_gca", "n_to_boris", "n_nonconv", "n_gcafail",
              "n_nonfinite", "sum_iter", "max_iter"):
        assert stats_a[k] == stats_b[k], k
    assert stats_a["sum_ekin"] == pytest.approx(stats_b["sum_ekin"], rel=RTOL)


@pytest.mark.parametrize("precision,sort_every", [("fp64", 0), ("mixed", 0), ("mixed", 2)])
def test_noalloc_matches_workspace_entry_two_calls(G, precision, sort_every):
    fields, st, p = inputs.reconnection_2d(nx=256, ny=128, n_particles=6000, seed=21)
    p = dict(p, gca_fixed_iters=5, sort_every=sort_every)
    grid = G.Grid(fields, dtype="f64" if precision == "fp64" else "f32")
    ref = G.State.from_numpy(st, precision=precision, with_pid=True)
    new = G.State.from_numpy(st, precision=precision, with_pid=True)
    gp = G.make_params(p)
    ws = G.Workspace(ref, grid, gp)
    for call in range(2):
        gp.step_index = 3 * call
        s_ref = G.push(ref, grid, gp, 3, workspace=ws)
        rc, s_new = noalloc_push(G, new, grid, gp, 3)
        assert rc == 0, G.lib().gcb_last_error()
        assert_same(by_pid(new.to_numpy()), by_pid(ref.to_numpy()), s_new, s_ref)
    assert s_ref["n_gca"] > 0


def test_noalloc_rejects_problems_beyond_its_array(G):
    fields, st, p = inputs.reconnection_2d(nx=256, ny=128, n_particles=40000, seed=22)
    grid = G.Grid(fields, dtype="f32")
    ds = G.State.from_numpy(st, precision="mixed")
    gp = G.make_params(p, sort_every=1)          # 40000 particles need ~2.8 MB to sort
    before = ds.to_numpy()
    rc, _ = noalloc_push(G, ds, grid, gp, 1)
    assert rc == 4 and b"more than the fixed" in G.lib().gcb_last_error()
    after = ds.to_numpy()
    assert np.array_equal(after["x"], before["x"])   # nothing ran
    rc, s = noalloc_push(G, ds, grid, G.make_params(p), 1)   # without sorting it fits
    assert rc == 0 and s["n_gca"] + s["n_boris"] == 40000
