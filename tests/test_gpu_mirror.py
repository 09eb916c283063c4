"""The mirror terms (gcb_params.mirror = GCB_MIRROR_ON: the grad-B drift and
the mirror force that Sec. 2.2 discards) on the GPU against the oracle's,
through the C ABI.

FP64: one step of the Harris workload (2D, gradients from W; coupled, and
forced onto the guiding-center branch for the magnetized species) and of the
3D current sheet (coupled: forcing its unmagnetized power-law particles onto
the guiding-center branch moves some of them tens of cells in one step,
across faces where the gradient of W jumps) reproduces the oracle's flags
where the switch margin exceeds 1e-12 and its state to a relative 1e-12; the
option changes the step well beyond that.  A magnetic bottle sampled on a 3D grid: 400 forced
guiding-center steps reproduce the oracle's orbit (the guiding center
bounces) to 1e-9.  Mixed path: within FP32 rounding of the oracle.  The
paths that do not carry the option refuse it.
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


@pytest.mark.parametrize("force", [0, 2])
def test_fp64_mirror_terms_match_oracle_2d(G, force):
    fields, st, p = inputs.harris_2d(n_per_species=512, seed=31)
    if force == 2:
        # guiding-center steps forced on the magnetized species only (|q/m| >=
        # 100): on the others the switch would take Boris, and the forced
        # step's sensitivity to rounding, not the implementation, sets the
        # agreement
        st = inputs.subset(st, np.nonzero((st["flags"] >> 6) >= 2)[0])
    p = dict(p, gca_fixed_iters=6, force=force, mirror=1)
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    got, ref, gs, os_, _ = run_both(G, fields, st, p)
    frac = assert_fp64_parity(got, ref, m, (128.0, 128.0), (1.0, 1.0))
    assert frac > 0.999 and gs["n_gca"] > 100
    for k in ("n_boris", "n_gca", "n_gcafail", "sum_iter"):
        assert gs[k] == os_[k], (k, gs[k], os_[k])
    # the option changes the guiding-center step well beyond the tolerance
    plain = copy_state(st)
    O.push_sr(plain, oracle_field(fields), oracle_params(dict(p, mirror=0)), 1)
    gca = (ref["flags"] & 1) == 0
    d = np.abs(plain["x"][:, gca] - ref["x"][:, gca]).max()
    du = np.abs(plain["u"][:, gca] - ref["u"][:, gca]).max()
    assert max(d, du) > 1e-8, (d, du)


def test_fp64_mirror_terms_match_oracle_3d(G):
    fields, st, p = inputs.current_sheet_3d(n=24, n_particles=3000, seed=32)
    p = dict(p, gca_fixed_iters=5, force=0, mirror=1)
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    got, ref, gs, os_, _ = run_both(G, fields, st, p)
    frac = assert_fp64_parity(got, ref, m, (24.0, 24.0, 24.0), (1.0, 1.0, 1.0))
    assert frac > 0.999 and gs["n_gca"] > 1000


def test_fp64_mirror_terms_match_oracle_gradient_records(G):
    """The reconnection field with gradient records (grad_mode GRID): grad |B|
    from the records' d_i B_j."""
    fields, st, p = inputs.reconnection_2d(nx=64, ny=32, n_particles=4096 + 37,
                                           omega_dt_max=50.0, seed=36)
    p = dict(p, gca_fixed_iters=5, mirror=1)
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    got, ref, gs, os_, _ = run_both(G, fields, st, p)
    frac = assert_fp64_parity(got, ref, m, (64.0, 32.0), (1.0, 1.0))
    assert frac > 0.999 and gs["n_gca"] > 1000


def bottle_grid(B0=1.0, L=12.0, n=(16, 16, 64)):
    """B_z = B0 (1 + s^2/L^2), B_x = -B0 x' s/L^2, B_y = -B0 y' s/L^2 about the
    axis x' = y' = 0 (x' = x - 8, y' = y - 8, s = z - 32), sampled on nodes."""
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(ny, dtype=float),
                          np.arange(nx, dtype=float), indexing="ij")
    xs, ys, s = x - 8.0, y - 8.0, z - 32.0
    Z = np.zeros((nz, ny, nx))
    B = [-B0 * xs * s / L ** 2, -B0 * ys * s / L ** 2, B0 * (1.0 + s * s / L ** 2)]
    return dict(E=[Z, Z, Z], B=B, dB=None, dx=(1.0, 1.0, 1.0))


def test_bottle_orbit_matches_oracle(G):
    fields = bottle_grid()
    rng = np.random.default_rng(33)
    n = 64
    upar = rng.uniform(0.3, 0.8, n)
    uperp = rng.uniform(0.8, 1.5, n)
    x = np.stack([np.full(n, 8.0) + rng.uniform(-0.2, 0.2, n),
                  np.full(n, 8.0) + rng.uniform(-0.2, 0.2, n), np.full(n, 32.0)])
    u = np.stack([uperp, np.zeros(n), upar])
    Gm = np.sqrt(1.0 + (u * u).sum(0))
    dt = 0.1
    st = dict(x=x, u=u, dxp=np.stack([np.zeros(n), np.zeros(n), dt * upar / Gm]),
              flags=np.zeros(n, dtype=np.uint8))
    p = dict(c=1.0, dt=dt, f_rho=0.4, f_E=1.0, dl=1.0, qm=(-200.0,), curvature=1, mu_mode=0,
             grad_mode=0, gca_max_iter=16, gca_fixed_iters=4, gca_tol=1e-7, force=2, mirror=1)
    got, ref, gs, os_, _ = run_both(G, fields, st, p, n_steps=400)
    assert gs["n_gca"] == 400 * n
    assert np.abs(got["x"] - ref["x"]).max() < 1e-9 * 64
    assert np.abs(got["u"] - ref["u"]).max() < 1e-9 * 2
    # guiding centers turned back (parallel momentum of the other sign) and
    # none got far past the exact bottle's mirror point |s| = L u_par/u_perp
    assert (np.sign(got["u"][2]) != np.sign(upar)).sum() > n // 4
    z_m = 12.0 * upar / uperp
    assert np.all(np.abs(got["x"][2] - 32.0) < 1.1 * z_m + 0.5)


def test_mixed_mirror_terms_close_to_oracle(G):
    fields, st, p = inputs.harris_2d(n_per_species=512, seed=34)
    p = dict(p, gca_fixed_iters=6, mirror=1)
    got, ref, gs, os_, _ = run_both(G, fields, st, p, precision="mixed", pos_mode="pair")
    same = got["flags"] == ref["flags"]
    assert same.mean() > 0.98
    d = np.abs(got["u"][:, same] - ref["u"][:, same]) / (np.linalg.norm(ref["u"][:, same], axis=0) + 1)
    assert np.quantile(d, 0.99) < 1e-4
    assert gs["n_gca"] > 100


def test_paths_without_the_mirror_terms_refuse_them(G):
    import torch
    fields, st, p = inputs.reconnection_2d(nx=32, ny=16, n_particles=64, seed=35)
    grid = G.Grid(fields, dtype="f32")
    ds = G.State.from_numpy(st, precision="mixed", pos_mode="pair")
    with pytest.raises(G.GcbError, match="EINVAL"):
        G.push(ds, grid, G.make_params(p, mirror=2), 1)
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.push(ds, grid, G.make_params(p, mirror=1, fuse_steps=4), 4)
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.push(ds, grid, G.make_params(p, mirror=1, drift_frame=1), 1)
    lam = torch.zeros((7, ds.n), dtype=torch.float32, device="cuda")
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.adjoint(ds, grid, G.make_params(p, mirror=1, gca_fixed_iters=4), 2, lam)
    kf, kst, kp = inputs.kerr_wald(nr=32, nth=24, n_particles=16, seed=3)
    kgrid = G.KsGrid(kf, kp["a"], kp["r_in"], kp["r_out"], dtype="f32")
    kds = G.State.from_numpy(kst, precision="fp64")
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.push_ks(kds, kgrid, G.make_params(kp, mirror=1), 1)
