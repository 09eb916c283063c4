"""Particle states left in pinned host memory (include/gcb.h: host-resident
particles): the push reads and writes them in place across the host link.
The results equal those of the same state in device memory bit for bit
(flat FP64 and mixed paths with sorting and particle ids, compared particle
by particle through the ids since the order inside a sort tile is not
specified; the covariant push), and arrays the device cannot reach at their
address (plain pageable host memory) are refused before any launch."""
import ctypes as C

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


@pytest.mark.parametrize("precision,pos_mode,gdt", [("fp64", "f64", "f64"),
                                                     ("mixed", "pair", "f32")])
def test_host_state_equals_device_state(G, precision, pos_mode, gdt):
    fields, st, p = inputs.reconnection_2d(nx=128, ny=64, n_particles=20000, seed=12)
    grid = G.Grid(fields, dtype=gdt)
    gp = G.make_params(p, sort_every=3, sort_tile=(1, 1))
    out = []
    for device in ("cuda", "pinned"):
        ds = G.State.from_numpy(st, precision=precision, pos_mode=pos_mode, device=device,
                                with_pid=True)
        assert ds.host == (device == "pinned") and ds.u.is_cuda == (device == "cuda")
        ws = G.Workspace(ds, grid, gp, device="cuda")
        s = None
        for k in range(7):
            gp.step_index = k
            s = G.push(ds, grid, gp, 1, workspace=ws)
        out.append((ds.to_numpy(), s))
    (a, sa), (b, sb) = out
    oa, ob = np.argsort(a["pid"]), np.argsort(b["pid"])
    for k in a:
        assert np.array_equal(a[k][..., oa], b[k][..., ob]), k
    # the kinetic-energy sum is reduced with atomics in an unspecified order
    assert {k: v for k, v in sa.items() if k != "sum_ekin"} == \
        {k: v for k, v in sb.items() if k != "sum_ekin"}
    assert sa["sum_ekin"] == pytest.approx(sb["sum_ekin"], rel=1e-12)


@pytest.mark.parametrize("n", [1, 31, 33, 4096 + 7])
@pytest.mark.parametrize("pos_mode", ["pair", "f64"])
def test_small_and_ragged_states_without_sorting(G, n, pos_mode):
    """Without sorting the push reads the caller's arrays: a device state
    through the shared-memory copies of the 2D mixed kernels' next tile, a
    host state with plain loads.  The two give the same state bit for bit,
    for one particle, a ragged single tile, a ragged second tile and many
    tiles per block."""
    fields, st, p = inputs.reconnection_2d(nx=64, ny=32, n_particles=n, seed=15)
    grid = G.Grid(fields, dtype="f32")
    gp = G.make_params(p)
    out = []
    for device in ("cuda", "pinned"):
        ds = G.State.from_numpy(st, precision="mixed", pos_mode=pos_mode, device=device)
        ws = G.Workspace(ds, grid, gp, device="cuda")
        for k in range(3):
            gp.step_index = k
            G.push(ds, grid, gp, 1, workspace=ws)
        out.append(ds.to_numpy())
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


def test_host_state_covariant(G):
    fields, st, p = inputs.kerr_wald(nr=64, nth=48, n_particles=3000, seed=13)
    grid = G.KsGrid(fields, p["a"], p["r_in"], p["r_out"], dtype="f32")
    res = []
    for device in ("cuda", "pinned"):
        ds = G.State.from_numpy(st, precision="fp64", device=device)
        G.push_ks(ds, grid, G.make_params(p), 5)
        res.append(ds.to_numpy())
    for k in res[0]:
        assert np.array_equal(res[0][k], res[1][k]), k


def test_unreachable_arrays_are_refused(G):
    """A state whose arrays are plain (pageable) host memory: every entry
    point refuses it before launching anything, and the arrays are left as
    they were."""
    fields, st, p = inputs.reconnection_2d(nx=32, ny=16, n_particles=256, seed=14)
    grid = G.Grid(fields, dtype="f32")
    ds = G.State.from_numpy(st, precision="mixed", pos_mode="pair")
    arrs = {k: t.cpu().numpy().copy() for k, t in
            (("x", ds.x), ("x_lo", ds.x_lo), ("u", ds.u), ("dxp", ds.dxp), ("flags", ds.flags))}
    s = G.GcbParticles()
    s.n, s.ndim, s.pos_mode, s.mom_dtype = ds.n, 2, G.POS_F32PAIR, G.F32
    for d in range(2):
        s.x[d] = arrs["x"][d].ctypes.data
        s.x_lo[d] = arrs["x_lo"][d].ctypes.data
        s.dxp[d] = arrs["dxp"][d].ctypes.data
    for k in range(3):
        s.u[k] = arrs["u"][k].ctypes.data
    s.flags = arrs["flags"].ctypes.data
    before = {k: v.copy() for k, v in arrs.items()}
    gp = G.make_params(p)
    ws = G.Workspace(ds, grid, gp)
    rc = G.lib().gcb_push_sr(C.byref(s), C.byref(grid.s), C.byref(gp), 1, None,
                             C.c_void_p(ws.buf.data_ptr()), ws.nbytes, None)
    assert rc == 1 and b"not reachable" in G.lib().gcb_last_error()
    rc = G.lib().gcb_pos_join(ds.n, C.c_void_p(arrs["x"][0].ctypes.data),
                              C.c_void_p(arrs["x_lo"][0].ctypes.data),
                              C.c_void_p(ds.x.data_ptr()), None)
    assert rc == 1
    for k in arrs:
        assert np.array_equal(arrs[k], before[k])
