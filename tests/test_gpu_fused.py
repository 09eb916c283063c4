"""The fused (test-particle) mode against one launch per step.

With fuse_steps = k the push takes up to k steps per kernel launch, keeping
each particle tile's state on chip between them; every step's arithmetic is
the same as in the one-launch-per-step mode, so after any number of steps every particle's
state and flags (matched by id) and the statistics must be identical bit for bit,
with and without sorting (a fused launch never spans a sort), and with a
particle that is frozen by a non-finite state.
"""
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


def run(G, fields, st, p, precision, gdt, n_steps, **over):
    grid = G.Grid(fields, dtype=gdt)
    ds = G.State.from_numpy(st, precision=precision, pos_mode="pair", with_pid=True)
    stats = G.push(ds, grid, G.make_params(p, **over), n_steps)
    return ds.to_numpy(), stats


def assert_identical(a, b):
    """Equal particle by particle (matched by id: the per-cell sort leaves the
    order of particles within a cell to its atomics, so it may differ)."""
    sa, ta = a
    sb, tb = b
    oa, ob = np.argsort(sa["pid"]), np.argsort(sb["pid"])
    np.testing.assert_array_equal(sa["pid"][oa], sb["pid"][ob])
    for k in ("x", "u", "dxp", "flags"):
        np.testing.assert_array_equal(sa[k][..., oa], sb[k][..., ob], err_msg=k)
    # integer counters exactly; the energy sum is accumulated in another order
    assert {k: v for k, v in ta.items() if k != "sum_ekin"} == \
        {k: v for k, v in tb.items() if k != "sum_ekin"}
    assert ta["sum_ekin"] == pytest.approx(tb["sum_ekin"], rel=1e-12)


CASES = {
    "harris_fp64": lambda: (inputs.harris_2d(n_per_species=512, seed=0), "fp64", "f64"),
    "reconnection_mixed": lambda: (inputs.reconnection_2d(nx=256, ny=128, n_particles=20000,
                                                          seed=5), "mixed", "f32"),
    "sheet3d_mixed": lambda: (inputs.current_sheet_3d(n=32, n_particles=12000, seed=6),
                              "mixed", "f32"),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("sort_every,fuse", [(0, 4), (0, 16), (3, 8), (5, 2)])
def test_fused_equals_stepwise(G, name, sort_every, fuse):
    (fields, st, p), precision, gdt = CASES[name]()
    n_steps = 10
    ref = run(G, fields, st, p, precision, gdt, n_steps, sort_every=sort_every, fuse_steps=0)
    got = run(G, fields, st, p, precision, gdt, n_steps, sort_every=sort_every,
              fuse_steps=fuse)
    assert_identical(got, ref)


def test_fused_with_frozen_particle(G):
    fields, st, p = inputs.harris_2d(n_per_species=256, seed=1)
    st = {k: v.copy() for k, v in st.items()}
    st["u"][1, 17] = np.nan
    ref = run(G, fields, st, p, "fp64", "f64", 6, fuse_steps=0)
    got = run(G, fields, st, p, "fp64", "f64", 6, fuse_steps=6)
    assert_identical(got, ref)
    assert got[0]["flags"][17] & 16
