"""Pushes captured in a CUDA graph (gcb.StepGraph) replay to the same results
as the same calls made one by one: bit for bit per particle for the FP64 and
mixed paths (with sorting, compared through the particle ids, the order
inside a sort tile being unspecified), over repeated replays, and with the
current deposited (to the rounding of the atomic additions' order)."""
import numpy as np
import pytest

from paper_2007_14401_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14401_gb300 import gcb
    return gcb


def _eager(G, ds, grid, gp, ws, steps, first, current=None):
    for k in steps:
        gp.step_index = first + k
        G.push(ds, grid, gp, 1, workspace=ws, stats=False, current=current)


@pytest.mark.parametrize("case", ["harris_fp64", "recon_mixed_sorted"])
def test_graph_replay_equals_eager_steps(G, case):
    import torch
    if case == "harris_fp64":
        fields, st, p = inputs.harris_2d(n_per_species=1024, seed=51)
        prec, pm, gdt, extra = "fp64", "f64", "f64", {}
    else:
        fields, st, p = inputs.reconnection_2d(nx=128, ny=64, n_particles=30000, seed=52)
        prec, pm, gdt, extra = "mixed", "pair", "f32", dict(sort_every=4, sort_tile=(1, 1))
    K = 8
    res = []
    for graphed in (False, True):
        grid = G.Grid(fields, dtype=gdt)
        ds = G.State.from_numpy(st, precision=prec, pos_mode=pm, with_pid=True)
        gp = G.make_params(p, **extra)
        ws = G.Workspace(ds, grid, gp)
        _eager(G, ds, grid, gp, ws, [0], 0)              # the kernels' first calls
        if graphed:
            gp.step_index = 1
            sg = G.StepGraph(ds, grid, gp, K, ws)
            sg.replay()
            sg.replay()
        else:
            _eager(G, ds, grid, gp, ws, list(range(K)) * 2, 1)
        torch.cuda.synchronize()
        res.append(ds.to_numpy())
    a, b = res
    oa, ob = np.argsort(a["pid"]), np.argsort(b["pid"])
    for k in a:
        assert np.array_equal(a[k][..., oa], b[k][..., ob]), k


def test_graph_with_deposition(G):
    import torch
    fields, st, p = inputs.reconnection_2d(nx=64, ny=32, n_particles=8192, seed=53,
                                           omega_dt_max=50.0)
    K = 4
    J = []
    for graphed in (False, True):
        grid = G.Grid(fields, dtype="f64")
        ds = G.State.from_numpy(st, precision="fp64", pos_mode="f64")
        gp = G.make_params(p)
        ws = G.Workspace(ds, grid, gp)
        cur = G.Current(grid, (-1.0, 1.0), precision="fp64")
        _eager(G, ds, grid, gp, ws, [0], 0, current=cur)
        cur.J.zero_()
        if graphed:
            gp.step_index = 1
            sg = G.StepGraph(ds, grid, gp, K, ws, current=cur)
            sg.replay()
        else:
            _eager(G, ds, grid, gp, ws, range(K), 1, current=cur)
        torch.cuda.synchronize()
        J.append(cur.J.cpu().numpy())
    scale = np.abs(J[0]).max()
    assert scale > 0 and np.abs(J[0] - J[1]).max() <= 1e-12 * scale
