"""Pins of the oracle's mirror terms (option mirror = 1; Sec. 2.2 names the
grad-B drift and the mirror force and discards them).  Reading: the grad-B
term (mu/(m Gamma)) grad(B)/kappa joins the bracket of the curvature drift
Eq. (curvdrift), and -(mu/(m Gamma)) b.grad(B)/kappa joins du_par/dt, the
force taken explicitly at (x^n, u_par^{n-1/2}).

- Magnetic bottle, E = 0: a guiding center on the axis bounces where
  B = B0 (1 + u_par0^2/u_perp0^2) (mu and Gamma conserved), i.e. at
  |z| = L u_par0/u_perp0; Gamma stays constant to the step's accuracy; with
  the option off it passes through.
- Uniform gradient B_z = B0 (1 + x/Lg), uniform E_x (E normal to B and to
  grad B): one step moves the guiding center along y by
  dt (-c E_x/B + c kappa mu (B0/Lg)/((q/m) B Gamma)), u_par unchanged, for
  both signs of the charge (the grad-B drift's direction, its kappa and its
  1/Gamma); a field tilted out of the plane, B parallel to (sin a, 0, cos a)
  with |B| growing along y, drifts along b x y-hat.
- Gradient along b, B_z = B0 (1 + z/Lg), E = 0: one step changes u_par by
  -dt mu (B0/Lg)/Gamma(x^n, u_par^{n-1/2}), with and without the curvature
  scheme.
"""
import math

import numpy as np
import pytest

import oracle as O


def _bottle_run(mirror, dt, n_steps, upar0=0.6, uperp0=1.2, B0=1.0, L=20.0):
    field = O.bottle_field(B0, L)
    p = O.make_params(dt=dt, qm=(-50.0,), force=O.FORCE_GCA, curvature=1, mirror=mirror,
                      tol=1e-12, max_iter=50)
    G = math.sqrt(1.0 + upar0 ** 2 + uperp0 ** 2)
    x = np.array([0.0, 0.0, 0.0])
    u = np.array([uperp0, 0.0, upar0])
    dxp = np.array([0.0, 0.0, dt * upar0 / G])
    zs, gs, ups = [], [], []
    for _ in range(n_steps):
        x, u, dxp, fl, det = O.step_one(field, p, x, u, dxp)
        assert det.branch == 0
        zs.append(x[2])
        gs.append(math.sqrt(1.0 + u @ u))
        ups.append(det.upar_new)
    return np.array(zs), np.array(gs), np.array(ups), G


def test_bottle_bounce_point_and_energy():
    upar0, uperp0, L = 0.6, 1.2, 20.0
    zs, gs, ups, G = _bottle_run(1, 0.05, 4000, upar0, uperp0, L=L)
    z_m = L * upar0 / uperp0
    assert zs.max() == pytest.approx(z_m, rel=2e-3)
    assert zs.min() == pytest.approx(-z_m, rel=2e-3)      # it comes back through the centre
    assert (ups < 0).any() and (ups > 0).any()
    assert np.abs(gs / G - 1.0).max() < 1e-3
    # the option off: u_par constant, the guiding center passes the mirror point
    zs0, _, ups0, _ = _bottle_run(0, 0.05, 1200, upar0, uperp0, L=L)
    assert np.allclose(ups0, upar0, rtol=0, atol=1e-12)
    assert zs0.max() > 1.5 * z_m


def _gradient_grid(E, Bz_of, ndim, n):
    shape = tuple(reversed(n))
    idx = np.indices(shape)
    coords = [idx[ndim - 1 - a].astype(float) for a in range(ndim)]    # node coordinates (dx = 1)
    Bz = Bz_of(*coords)
    z = np.zeros(shape)
    return O.grid_field([z + E[0], z + E[1], z + E[2]], [z, z, Bz], (1.0,) * ndim), coords


@pytest.mark.parametrize("qm", [-20.0, 30.0])
@pytest.mark.parametrize("E0", [0.0, 0.3])
def test_grad_B_drift_one_step(qm, E0):
    B0, Lg, dt = 1.0, 40.0, 0.4
    field, _ = _gradient_grid((E0, 0.0, 0.0), lambda x, y: B0 * (1.0 + x / Lg), 2, (32, 16))
    x0 = np.array([10.3, 7.6])
    u = np.array([0.5, -0.4, 0.0])                      # u_par = u_z = 0
    p = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_GCA, curvature=1, mirror=1,
                      fixed_iters=4)
    xo, uo, dxo, fl, det = O.step_one(field, p, x0.copy(), u.copy(), np.zeros(2))
    assert det.branch == 0
    B = B0 * (1.0 + x0[0] / Lg)
    vE = np.array([0.0, -E0 / B, 0.0])
    kappa = 1.0 / math.sqrt(1.0 - vE @ vE)
    Gfull = math.sqrt(1.0 + u @ u)
    ug = u - vE * Gfull
    mu = (ug @ ug) / (2.0 * B * kappa)
    Gam = kappa * math.sqrt(1.0 + 2.0 * mu * B * kappa)
    vy = -E0 / B + kappa * mu * (B0 / Lg) / (qm * B * Gam)
    assert dxo[0] == pytest.approx(0.0, abs=1e-13)
    assert dxo[1] == pytest.approx(dt * vy, rel=1e-12, abs=1e-15)
    assert det.upar_new == pytest.approx(0.0, abs=1e-14)
    # without the option only the E x B drift remains
    p0 = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_GCA, curvature=1, mirror=0,
                       fixed_iters=4)
    _, _, dx0, _, _ = O.step_one(field, p0, x0.copy(), u.copy(), np.zeros(2))
    assert dx0[1] == pytest.approx(-dt * E0 / B, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("alpha", [0.0, 0.7])
def test_grad_B_drift_tilted_field(alpha):
    """B = B0 (1 + y/Lg)(sin a, 0, cos a), E = 0: grad|B| = (0, B0/Lg, 0), the
    drift along b x y-hat = (-cos a, 0, sin a), whose x component moves the
    guiding center in the plane."""
    B0, Lg, dt, qm = 1.0, 25.0, 0.4, 15.0
    n = (16, 32)
    shape = tuple(reversed(n))
    y = np.indices(shape)[0].astype(float)
    mag = B0 * (1.0 + y / Lg)
    z = np.zeros(shape)
    field = O.grid_field([z, z, z], [math.sin(alpha) * mag, z, math.cos(alpha) * mag],
                         (1.0, 1.0))
    x0 = np.array([7.4, 12.2])
    b = np.array([math.sin(alpha), 0.0, math.cos(alpha)])
    u = np.array([0.6 * math.cos(alpha), 0.5, -0.6 * math.sin(alpha)])   # u . b = 0
    p = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_GCA, curvature=1, mirror=1,
                      fixed_iters=4)
    _, _, dxo, _, det = O.step_one(field, p, x0.copy(), u.copy(), np.zeros(2))
    assert det.branch == 0 and abs(u @ b) < 1e-15
    B = B0 * (1.0 + x0[1] / Lg)
    mu = (u @ u) / (2.0 * B)
    Gam = math.sqrt(1.0 + 2.0 * mu * B)
    vx = -math.cos(alpha) * mu * (B0 / Lg) / (qm * B * Gam)
    assert dxo[0] == pytest.approx(dt * vx, rel=1e-12)
    assert dxo[1] == pytest.approx(0.0, abs=1e-13)


@pytest.mark.parametrize("curvature", [0, 1])
def test_mirror_force_one_step(curvature):
    B0, Lg, dt = 1.0, 30.0, 0.3
    field, _ = _gradient_grid((0.0, 0.0, 0.0), lambda x, y, z: B0 * (1.0 + z / Lg), 3,
                              (8, 8, 24))
    x0 = np.array([3.2, 4.1, 9.7])
    u = np.array([0.8, 0.3, 0.9])
    G = math.sqrt(1.0 + u @ u)
    dxp = np.array([0.0, 0.0, dt * u[2] / G])
    p = O.make_params(dt=dt, qm=(-100.0,), force=O.FORCE_GCA, curvature=curvature, mirror=1,
                      fixed_iters=3)
    _, _, _, _, det = O.step_one(field, p, x0.copy(), u.copy(), dxp.copy())
    assert det.branch == 0
    # mu from the conversion at R^{n-1/2} = x^n - dxp/2, the force at x^n
    Bh = B0 * (1.0 + (x0[2] - 0.5 * dxp[2]) / Lg)
    mu = (u[0] ** 2 + u[1] ** 2) / (2.0 * Bh)
    Bn = B0 * (1.0 + x0[2] / Lg)
    G0 = math.sqrt(1.0 + u[2] ** 2 + 2.0 * mu * Bn)
    assert det.mu == pytest.approx(mu, rel=1e-13)
    assert det.upar_new == pytest.approx(u[2] - dt * mu * (B0 / Lg) / G0, rel=1e-13)
