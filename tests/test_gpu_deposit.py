"""Current deposition (gcb_push_deposit_sr: the PiC coupling of the coupled
push) on the GPU against the oracle's deposition, through the C ABI.

Parity: from identical states (restricted to particles whose flags the two
sides agree on and whose switch margin is clear of rounding), one step of
each side deposits J on every staggered point within
  FP64:  1e-11 x (sum of |contributions| at that point) + 1e-14 x max|J|,
  mixed: 1e-4  x (sum of |contributions| at that point) + 1e-7  x max|J|
(the atomic additions run in an unspecified order; the mixed path's
per-particle displacements carry FP32 rounding).  Cases: 2D reconnection
and 3D current sheet in both precisions (several tiles and a ragged tail),
forced branches, two species with charges and weights, sorting, fields that
change between steps (grid.update), paths longer than the cap, non-finite
particles, an empty state, the step's options (the mirror terms, the exact
drift frame).  At the full 2D size of the benchmark: the
discrete continuity equation with the cloud-in-cell charge of the positions
before and after the step, and the total current against the particles' own
displacements.  Option combinations the push does not carry (fused steps,
the mirror terms in the exact frame, the exact frame with FP64 positions on
the mixed path) are refused.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_14401_gb300 import inputs
from tests.helpers import oracle_field, oracle_params, switch_margins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14401_gb300 import gcb
    return gcb


TOL = {"fp64": (1e-11, 1e-14), "mixed": (1e-4, 1e-7)}


def agreeing_subset(G, fields, st, p, precision, pos_mode, margin_min):
    """Indices of the particles whose one-step flags agree between the GPU
    and the oracle and whose switch margin exceeds margin_min."""
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    grid = G.Grid(fields, dtype="f64" if precision == "fp64" else "f32")
    ds = G.State.from_numpy(st, precision=precision, pos_mode=pos_mode)
    G.push(ds, grid, G.make_params(p), 1)
    got = ds.to_numpy()
    ref = {k: v.copy() for k, v in st.items()}
    O.push_sr(ref, oracle_field(fields), oracle_params(p), 1)
    keep = (got["flags"] == ref["flags"]) & (np.abs(m) > margin_min)
    return np.nonzero(keep)[0]


def deposit_both(G, fields, st, p, precision, pos_mode, q, w=None, n_steps=1, fields2=None,
                 **over):
    gdt = "f64" if precision == "fp64" else "f32"
    grid = G.Grid(fields, dtype=gdt)
    ds = G.State.from_numpy(st, precision=precision, pos_mode=pos_mode)
    gp = G.make_params(p, **over)
    cur = G.Current(grid, q, precision=precision, w=w)
    G.push(ds, grid, gp, n_steps, current=cur)
    ref = {k: v.copy() for k, v in st.items()}
    ocur = O.Current(grid.shape, q=q, w=w)
    O.push_sr(ref, oracle_field(fields), oracle_params(p, **over), n_steps, current=ocur)
    if fields2 is not None:
        grid.update(fields2)
        G.push(ds, grid, gp, 1, current=cur)
        O.push_sr(ref, oracle_field(fields2), oracle_params(p, **over), 1, current=ocur)
    return cur, ocur, ds, ref


def assert_current_parity(cur, ocur, precision):
    rel, floor = TOL[precision]
    J = cur.J.double().cpu().numpy()
    scale = max(np.abs(ocur.J[a]).max() for a in range(3)) + 1e-300
    for a in range(3):
        err = np.abs(J[a] - ocur.J[a])
        lim = rel * ocur.Jabs[a] + floor * scale
        assert np.all(err <= lim), (a, float((err / (ocur.Jabs[a] + floor * scale)).max()))
    assert cur.n_skipped == ocur.n_skipped


def recon(n=4096 + 37, seed=21):
    return inputs.reconnection_2d(nx=64, ny=32, n_particles=n, omega_dt_max=50.0, seed=seed)


def sheet(n=3000 + 19, seed=22):
    return inputs.current_sheet_3d(n=24, n_particles=n, seed=seed)


@pytest.mark.parametrize("precision,pos_mode", [("fp64", "f64"), ("mixed", "pair"),
                                                ("mixed", "f64")])
@pytest.mark.parametrize("workload", ["recon2d", "sheet3d"])
def test_one_step_current_matches_oracle(G, precision, pos_mode, workload):
    fields, st, p = recon() if workload == "recon2d" else sheet()
    p = dict(p, gca_fixed_iters=5)
    idx = agreeing_subset(G, fields, st, p, precision, pos_mode,
                          1e-12 if precision == "fp64" else 1e-4)
    assert idx.size > 0.95 * st["flags"].size
    sub = inputs.subset(st, idx)
    cur, ocur, ds, ref = deposit_both(G, fields, sub, p, precision, pos_mode, q=(-1.0, 1.0))
    assert_current_parity(cur, ocur, precision)
    assert np.abs(ocur.J[0]).max() > 0 and np.abs(ocur.J[2]).max() > 0
    # one piece per particle-step plus one per cell face crossed (from the
    # positions before and the displacement of the step)
    dx = np.asarray(fields["dx"])[:, None]
    s0 = sub["x"] / dx
    s1 = s0 + ref["dxp"] / dx
    want = sub["flags"].size + int(np.abs(np.floor(s1) - np.floor(s0)).sum())
    assert abs(cur.n_pieces - want) <= (0 if precision == "fp64" else 1e-3 * want)
    slots = 8 if len(fields["dx"]) == 2 else 12
    assert cur.n_pieces <= cur.n_atomics <= slots * cur.n_pieces


@pytest.mark.parametrize("force", [1, 2])
def test_forced_branches(G, force):
    fields, st, p = recon(seed=23)
    p = dict(p, gca_fixed_iters=5, force=force)
    idx = agreeing_subset(G, fields, st, p, "fp64", "f64", 0.0)
    sub = inputs.subset(st, idx)
    cur, ocur, _, _ = deposit_both(G, fields, sub, p, "fp64", "f64", q=(-2.0, 3.0))
    assert_current_parity(cur, ocur, "fp64")


@pytest.mark.parametrize("precision,pos_mode", [("fp64", "f64"), ("mixed", "pair")])
def test_weights_and_changing_fields(G, precision, pos_mode):
    """Per-particle weights, two species charges, and a second step in fields
    repacked in place (the field a PiC code hands the next push)."""
    fields, st, p = recon(seed=24)
    p = dict(p, gca_fixed_iters=5)
    f2 = {k: v for k, v in fields.items()}
    f2["E"] = [1.5 * e for e in fields["E"]]
    f2["B"] = [0.9 * b for b in fields["B"]]
    f2["dB"] = [0.9 * d for d in fields["dB"]]
    idx = agreeing_subset(G, fields, st, p, precision, pos_mode,
                          1e-12 if precision == "fp64" else 1e-4)
    sub = inputs.subset(st, idx)
    # the second step's flags must agree as well: keep those of the first
    # step's survivors whose second step agrees
    grid = G.Grid(fields, dtype="f64" if precision == "fp64" else "f32")
    ds = G.State.from_numpy(sub, precision=precision, pos_mode=pos_mode)
    G.push(ds, grid, G.make_params(p), 1)
    mid = ds.to_numpy()
    idx2 = agreeing_subset(G, f2, mid, p, precision, pos_mode,
                           1e-12 if precision == "fp64" else 1e-4)
    sub = inputs.subset(sub, idx2)
    rng = np.random.default_rng(3)
    w = rng.uniform(0.2, 2.0, sub["flags"].size)
    cur, ocur, _, _ = deposit_both(G, fields, sub, p, precision, pos_mode, q=(-1.0, 0.5), w=w,
                                   fields2=f2)
    assert_current_parity(cur, ocur, precision)


def test_several_steps_in_one_call_and_host_state(G):
    """Three steps in one call add the three steps' currents (against the
    oracle's three steps); a state left in pinned host memory deposits the
    same current as the same state on the device."""
    import torch
    fields, st, p = recon(n=2048 + 5, seed=27)
    p = dict(p, gca_fixed_iters=5, force=1)
    cur, ocur, ds, ref = deposit_both(G, fields, st, p, "fp64", "f64", q=(-1.0, 1.0), n_steps=3)
    assert_current_parity(cur, ocur, "fp64")
    grid = G.Grid(fields, dtype="f64")
    J = []
    for device in ("cuda", "pinned"):
        s = G.State.from_numpy(st, precision="fp64", pos_mode="f64", device=device)
        c = G.Current(grid, (-1.0, 1.0), precision="fp64")
        G.push(s, grid, G.make_params(p), 2, current=c)
        torch.cuda.synchronize()
        J.append(c.J.cpu().numpy())
    scale = np.abs(J[0]).max()
    assert scale > 0 and np.abs(J[0] - J[1]).max() <= 1e-12 * scale


@pytest.mark.parametrize("option", ["mirror", "exact_frame"])
@pytest.mark.parametrize("precision,pos_mode", [("fp64", "f64"), ("mixed", "pair")])
def test_current_with_step_options(G, option, precision, pos_mode):
    """The deposition follows the step with its options: the mirror terms
    (reconnection field) and the exact drift frame (Harris sheet with a guide
    field and E.B != 0); either changes the oracle's current by percents."""
    if option == "mirror":
        fields, st, p = recon(seed=28)
        over = dict(mirror=1)
    else:
        fields, st, p = inputs.harris_2d(n_per_species=2048, seed=29, Bg=0.3, Ez=0.08)
        over = dict(drift_frame=O.FRAME_BT)
    p = dict(p, gca_fixed_iters=5, **over)
    idx = agreeing_subset(G, fields, st, p, precision, pos_mode,
                          1e-12 if precision == "fp64" else 1e-4)
    assert idx.size > 0.95 * st["flags"].size
    sub = inputs.subset(st, idx)
    cur, ocur, _, _ = deposit_both(G, fields, sub, p, precision, pos_mode, q=(-1.0, 1.0))
    assert_current_parity(cur, ocur, precision)
    plain = O.Current(cur.J.shape[1:], q=(-1.0, 1.0))
    O.push_sr({k: v.copy() for k, v in sub.items()}, oracle_field(fields),
              oracle_params(dict(p, mirror=0, drift_frame=O.FRAME_SIMPLE)), 1, current=plain)
    J0, J1 = np.array(ocur.J), np.array(plain.J)
    assert np.abs(J0 - J1).max() > 1e-2 * np.abs(J0).max()


def test_sorting_does_not_change_the_current(G):
    fields, st, p = recon(seed=25)
    p = dict(p, gca_fixed_iters=5)
    idx = agreeing_subset(G, fields, st, p, "fp64", "f64", 1e-12)
    sub = inputs.subset(st, idx)
    cur, ocur, _, _ = deposit_both(G, fields, sub, p, "fp64", "f64", q=(-1.0, 1.0),
                                   sort_every=1, sort_tile=(4, 4))
    assert_current_parity(cur, ocur, "fp64")


def test_long_paths_nonfinite_and_empty(G):
    """A Boris step with c dt = 100 cells: particles faster than 0.64 c move
    more than the cap and are left out and counted on both sides; a
    non-finite particle deposits nothing; an empty state leaves J as it was."""
    nx, ny = 32, 16
    one = np.ones((ny, nx))
    fields = dict(E=[0 * one] * 3, B=[0 * one, 0 * one, 0.01 * one], dB=[0 * one] * 6,
                  dx=(1.0, 1.0))
    rng = np.random.default_rng(4)
    n = 300
    u = rng.normal(0, 1.0, (3, n))
    x = np.stack([rng.uniform(0, nx, n), rng.uniform(0, ny, n)])
    st = dict(x=x, u=u, dxp=np.zeros((2, n)), flags=np.zeros(n, dtype=np.uint8))
    st["u"][0, 7] = np.nan
    p = dict(c=1.0, dt=100.0, f_rho=0.4, f_E=1.0, dl=1.0, qm=(-1.0,), curvature=1, mu_mode=0,
             grad_mode=1, gca_max_iter=16, gca_fixed_iters=3, gca_tol=1e-7, force=1)
    cur, ocur, ds, ref = deposit_both(G, fields, st, p, "fp64", "f64", q=(1.0,))
    assert ocur.n_skipped > 10 and ocur.n_skipped < n - 10
    assert_current_parity(cur, ocur, "fp64")
    e = inputs.subset(st, np.array([], dtype=np.int64))
    grid = G.Grid(fields, dtype="f64")
    c0 = G.Current(grid, (1.0,), precision="fp64")
    c0.J.fill_(2.5)
    G.push(G.State.from_numpy(e, precision="fp64"), grid, G.make_params(p), 1, current=c0)
    assert bool((c0.J == 2.5).all()) and c0.n_skipped == 0


@pytest.mark.parametrize("workload", ["recon2d", "sheet3d"])
def test_full_size_continuity_and_total(G, workload):
    """The benchmark's workloads at full size (2D: 2^24 particles, 2048 x 1024
    nodes; 3D: 2^26 particles, 256^3 nodes), mixed path, one step with
    deposition in the benchmark's sorted order: (rho^{n+1} - rho^n)/dt +
    div J = 0 with the cloud-in-cell charge of the positions before and after
    (FP64 on the device), and sum J_a V = sum q w dxp_a/dt over the
    particles."""
    import torch
    if workload == "recon2d":
        fields, st, p = inputs.reconnection_2d(seed=1)
        tile = (1, 1)
    else:
        fields, st, p = inputs.current_sheet_3d(seed=2)
        tile = (1, 1, 1)
    grid = G.Grid(fields, dtype="f32")
    nd = grid.ndim
    ds = G.State.from_numpy(st, precision="mixed", pos_mode="pair")
    G.sort(ds, grid, G.make_params(p, sort_every=1, sort_tile=tile))
    x0 = torch.as_tensor(ds.to_numpy()["x"]).cuda()
    sp = ds.flags.to(torch.int64) >> 6
    q = torch.where(sp == 0, -1.0, 1.0).double()
    cur = G.Current(grid, (-1.0, 1.0), precision="mixed")
    s = G.push(ds, grid, G.make_params(p), 1, current=cur)
    x1 = torch.as_tensor(ds.to_numpy()["x"]).cuda()
    n = grid.n[:nd]
    dt = p["dt"]
    r0, r1 = cic_rho_torch(x0, q, n), cic_rho_torch(x1, q, n)
    del x0, x1
    J = cur.J.double()
    div = torch.zeros_like(r0)
    for a in range(nd):
        div += J[a] - torch.roll(J[a], 1, dims=nd - 1 - a)
    res = (r1 - r0) / dt + div
    scale = max(float(J[:nd].abs().max()), float(r0.abs().max()) / dt)
    assert float(res.abs().max()) < 1e-4 * scale, (float(res.abs().max()), scale)
    dxp = ds.dxp.double()
    for a in range(nd):
        tot = float((q * dxp[a]).sum()) / dt
        tot_abs = float((q * dxp[a]).abs().sum()) / dt
        assert abs(float(J[a].sum()) - tot) <= 1e-5 * tot_abs
    assert s["n_nonfinite"] == 0 and cur.n_skipped == 0


def cic_rho_torch(x, q, n):
    """Cloud-in-cell charge at the nodes (unit cells, periodic), FP64."""
    import torch
    nd = len(n)
    base = [torch.floor(x[a]).long() for a in range(nd)]
    frac = [x[a] - base[a] for a in range(nd)]
    size = 1
    for v in n:
        size *= v
    rho = torch.zeros(size, dtype=torch.float64, device=x.device)
    for o in range(1 << nd):
        w = q.clone()
        idx = torch.zeros_like(base[0])
        stride = 1
        for a in range(nd):
            off = (o >> a) & 1
            w = w * (frac[a] if off else 1 - frac[a])
            idx += ((base[a] + off) % n[a]) * stride
            stride *= n[a]
        rho.index_add_(0, idx, w)
    return rho.view(*reversed(n))


def test_refused_options(G):
    import torch
    fields, st, p = recon(n=64, seed=26)
    grid = G.Grid(fields, dtype="f32")
    ds = G.State.from_numpy(st, precision="mixed", pos_mode="pair")
    cur = G.Current(grid, (-1.0, 1.0), precision="mixed")
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.push(ds, grid, G.make_params(p, fuse_steps=4), 4, current=cur)
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.push(ds, grid, G.make_params(p, drift_frame=1, mirror=1), 1, current=cur)
    f64 = G.State.from_numpy(st, precision="mixed", pos_mode="f64")
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.push(f64, grid, G.make_params(p, drift_frame=1), 1, current=cur)
    wc = G.Current(grid, (-1.0, 1.0), precision="mixed", w=np.ones(ds.n))
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.push(ds, grid, G.make_params(p, sort_every=1), 1, current=wc)
    bad = G.Current(grid, (-1.0, 1.0), precision="fp64")
    with pytest.raises(G.GcbError, match="EINVAL"):
        G.push(ds, grid, G.make_params(p), 1, current=bad)
    nan = G.Current(grid, (float("nan"), 1.0), precision="mixed")
    with pytest.raises(G.GcbError, match="EINVAL"):
        G.push(ds, grid, G.make_params(p), 1, current=nan)
    assert float(cur.J.abs().sum()) == 0.0
