"""The cell-tile sort: a permutation (ids follow), tiles in order, and no
effect on any particle's result (each particle's arithmetic does not depend
on where it sits in the arrays)."""
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


def tile_key(x, dx, n, tile):
    key = np.zeros(x.shape[1], dtype=np.int64)
    mul = 1
    for d in range(x.shape[0]):
        c = np.clip(np.floor(x[d] / dx[d]).astype(np.int64), 0, n[d] - 1)
        key += (c // tile[d]) * mul
        mul *= -(-n[d] // tile[d])
    return key


@pytest.mark.parametrize("precision,pos_mode,tile", [("mixed", "pair", (16, 8)),
                                                     ("mixed", "f64", (1, 1)),
                                                     ("fp64", "f64", (2, 4))])
def test_sort_is_a_tile_ordered_permutation(G, precision, pos_mode, tile):
    fields, st, p = inputs.reconnection_2d(nx=256, ny=128, n_particles=50001, seed=2)
    st["x"][0, 17] = np.nan          # non-finite positions go last
    grid = G.Grid(fields, dtype="f32" if precision == "mixed" else "f64")
    ds = G.State.from_numpy(st, precision=precision, pos_mode=pos_mode, with_pid=True)
    gp = G.make_params(p, sort_every=1, sort_tile=tile + (1,))
    before = ds.to_numpy()
    G.sort(ds, grid, gp)
    after = ds.to_numpy()
    pid = after["pid"]
    assert np.array_equal(np.sort(pid), np.arange(st["flags"].size))
    for k in ("x", "u", "dxp", "flags"):
        assert np.array_equal(after[k], before[k][..., pid], equal_nan=(k != "flags"))
    fin = np.isfinite(after["x"]).all(0) & np.isfinite(after["u"]).all(0)
    key = tile_key(after["x"][:, fin], (1.0, 1.0), (256, 128), tile)
    assert np.all(np.diff(key) >= 0)
    assert pid[-1] == 17 and fin[:-1].all()


def test_push_with_sorting_matches_push_without(G):
    fields, st, p = inputs.reconnection_2d(nx=256, ny=128, n_particles=40000, seed=3)
    grid = G.Grid(fields, dtype="f32")
    res = []
    for sort_every in (0, 3):
        ds = G.State.from_numpy(st, precision="mixed", pos_mode="pair", with_pid=True)
        gp = G.make_params(p, sort_every=sort_every, step_index=0)
        ws = G.Workspace(ds, grid, gp)
        s = G.push(ds, grid, gp, 7, workspace=ws)
        out = ds.to_numpy()
        order = np.argsort(out["pid"])
        res.append(({k: v[..., order] for k, v in out.items()}, s))
    (a, sa), (b, sb) = res
    for k in ("x", "u", "dxp", "flags"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("n_boris", "n_gca", "sum_iter", "max_iter", "n_nonconv"):
        assert sa[k] == sb[k]
    assert sa["sum_ekin"] == pytest.approx(sb["sum_ekin"], rel=1e-12)


def test_sort_needs_workspace(G):
    fields, st, p = inputs.reconnection_2d(nx=64, ny=32, n_particles=1000, seed=4)
    grid = G.Grid(fields, dtype="f32")
    ds = G.State.from_numpy(st, precision="mixed")
    gp = G.make_params(p, sort_every=1)
    small = G.Workspace(ds, grid, G.make_params(p))   # sized without sorting
    with pytest.raises(G.GcbError, match="ENOMEM"):
        G.push(ds, grid, gp, 1, workspace=small)
