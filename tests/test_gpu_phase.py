"""The evolved gyration phase (gcb_params.gyro_phase = GCB_PHASE_EVOLVE) on the
GPU against the oracle's, through the C ABI.

FP64: one step of the Harris workload (q/m = -1 and -10, so the step's
gyro-phase stays below ~50 rad and its rounding below the parity tolerance:
the angle's relative rounding becomes an absolute phase error proportional to
Omega_C dt) reproduces the oracle's flags where the switch margin exceeds
1e-12 and its state to a relative 1e-12; in uniform B with E = 0 the
guiding-center step reproduces the exact gyration of the Lorentz force over
many steps at Omega_C dt = 300 (FP64 to 1e-11; the mixed path to the phase
error its FP32 inputs give the angle, Omega_C dt x 1e-7 a step).  The
covariant push and the adjoint refuse the option.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2007_14401_gb300 import inputs
from tests.helpers import oracle_field, oracle_params, switch_margins
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
def test_fp64_evolved_phase_matches_oracle(G, force):
    fields, st, p = inputs.harris_2d(n_per_species=1024, seed=9, qms=(-1.0, -10.0))
    p = dict(p, gca_fixed_iters=6, force=force, gyro_phase=1)
    m = switch_margins(oracle_field(fields), oracle_params(p), st)
    got, ref, gs, os_, _ = run_both(G, fields, st, p)
    frac = assert_fp64_parity(got, ref, m, (128.0, 128.0), (1.0, 1.0))
    assert frac > 0.999 and gs["n_gca"] > 100
    for k in ("n_boris", "n_gca", "n_gcafail", "sum_iter"):
        assert gs[k] == os_[k], (k, gs[k], os_[k])


# the mixed path takes the angle from FP32 B, kappa and Gamma: its phase
# error is Omega_C dt times the FP32 rounding, ~3e-5 rad a step here
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 5e-3)])
def test_uniform_B_exact_gyration(G, precision, tol):
    nx, ny = 16, 8
    one = np.ones((ny, nx))
    zero = 0.0 * one
    B0, qm, n_steps = 1.5, -40.0, 12
    fields = dict(E=[zero, zero, zero], B=[zero, zero, B0 * one], dB=[zero] * 6, dx=(1.0, 1.0))
    rng = np.random.default_rng(10)
    n = 256
    u0 = rng.standard_normal((3, n)) * 0.5
    x0 = np.stack([rng.uniform(0, nx, n), rng.uniform(0, ny, n)])
    st = dict(x=x0, u=u0.copy(), dxp=np.zeros((2, n)), flags=np.zeros(n, dtype=np.uint8))
    G_ = np.sqrt(1.0 + (u0 * u0).sum(0))
    dt = 300.0 * np.median(G_) / (abs(qm) * B0)
    p = dict(c=1.0, dt=dt, f_rho=0.4, f_E=1.0, dl=1.0, qm=(qm,), curvature=1, mu_mode=0,
             grad_mode=1, gca_max_iter=16, gca_fixed_iters=3, gca_tol=1e-7, force=2,
             gyro_phase=1)
    grid = G.Grid(fields, dtype="f64" if precision == "fp64" else "f32")
    ds = G.State.from_numpy(st, precision=precision, pos_mode="pair")
    G.push(ds, grid, G.make_params(p), n_steps)
    got = ds.to_numpy()
    a = -qm * B0 * n_steps * dt / G_
    c, s = np.cos(a), np.sin(a)
    want = np.stack([c * u0[0] - s * u0[1], s * u0[0] + c * u0[1], u0[2]])
    err = np.abs(got["u"] - want).max(0) / G_
    assert err.max() < tol, err.max()


def test_paths_without_the_evolved_phase_refuse_it(G):
    import torch
    fields, st, p = inputs.reconnection_2d(nx=32, ny=16, n_particles=64, seed=8)
    grid = G.Grid(fields, dtype="f32")
    ds = G.State.from_numpy(st, precision="mixed", pos_mode="pair")
    with pytest.raises(G.GcbError, match="EINVAL"):
        G.push(ds, grid, G.make_params(p, gyro_phase=3), 1)
    lam = torch.zeros((7, ds.n), dtype=torch.float32, device="cuda")
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.adjoint(ds, grid, G.make_params(p, gyro_phase=1, gca_fixed_iters=4), 2, lam)
    kf, kst, kp = inputs.kerr_wald(nr=32, nth=24, n_particles=16, seed=3)
    kgrid = G.KsGrid(kf, kp["a"], kp["r_in"], kp["r_out"], dtype="f32")
    kds = G.State.from_numpy(kst, precision="fp64")
    with pytest.raises(G.GcbError, match="UNSUPPORTED"):
        G.push_ks(kds, kgrid, G.make_params(kp, gyro_phase=1), 1)
