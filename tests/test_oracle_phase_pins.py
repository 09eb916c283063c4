"""Pins of the oracle's evolved gyration phase (gyro_phase = 1; Sec. 3.1 keeps
the direction of u_perp,g and notes that the phase could be evolved by an
extra equation): the gyration direction turns about b by
phi = -(q/m) B dt / (c kappa Gamma) per guiding-center step.

- Uniform B, E = 0: the guiding-center step with the evolved phase
  reproduces the exact gyration of the Lorentz force, du/dt = (q/(m Gamma c))
  u x B (u_perp turns about B by -(q/m) B t/(c Gamma), u_par and |u_perp|
  fixed), at any Omega_C dt; without it the momentum stays frozen.
- Uniform E normal to B: one step turns the gyration direction (taken normal
  to v_E, so the decomposition is exact) by phi with the drift frame's
  kappa, and in the sense set by the sign of the charge.
"""
import math

import numpy as np
import pytest

import oracle as O


def rot_z(v, a):
    c, s = math.cos(a), math.sin(a)
    return np.array([c * v[0] - s * v[1], s * v[0] + c * v[1], v[2]])


@pytest.mark.parametrize("qm,omega_dt", [(-2.0, 0.3), (5.0, 7.0), (-40.0, 300.0)])
def test_uniform_B_exact_gyration(qm, omega_dt):
    B0 = 1.5
    u0 = np.array([0.6, -0.2, 0.4])
    G = math.sqrt(1.0 + u0 @ u0)
    dt = omega_dt * G / (abs(qm) * B0)
    field = O.uniform_field((0.0, 0.0, 0.0), (0.0, 0.0, B0), ndim=2)
    p = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_GCA, fixed_iters=3, gyro_phase=1,
                      curvature=1)
    x, u, dxp = np.array([1.0, 2.0]), u0.copy(), np.zeros(2)
    n = 9
    for _ in range(n):
        x, u, dxp, fl, det = O.step_one(field, p, x, u, dxp)
        assert det.branch == 0
    want = rot_z(u0, -qm * B0 * n * dt / G)
    assert np.allclose(u, want, rtol=0, atol=1e-12 * G)
    p0 = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_GCA, fixed_iters=3, gyro_phase=0)
    xf, uf, _, _, _ = O.step_one(field, p0, np.array([1.0, 2.0]), u0.copy(), np.zeros(2))
    assert np.allclose(uf, u0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("qm", [-3.0, 4.0])
def test_drift_frame_rate_and_sense(qm):
    """E = E_y y-hat, B = B_z z-hat (v_E along x, kappa > 1); u = v_E Gamma +
    u_perp b_perp with b_perp = b x v_E/|v_E| (normal to v_E and b): one step
    turns b_perp about b by -(q/m) B dt/(c kappa Gamma)."""
    Ey, Bz, dt = 0.4, 1.0, 0.7
    vE = np.array([Ey / Bz, 0.0, 0.0])
    kappa = 1.0 / math.sqrt(1.0 - vE @ vE)
    bp = np.array([0.0, 1.0, 0.0])                 # z x x-hat
    up = 0.8
    Gam = kappa * math.sqrt(1.0 + up * up)         # Eq. lfacgca2 with u_par = 0
    u = vE * Gam + up * bp
    field = O.uniform_field((0.0, Ey, 0.0), (0.0, 0.0, Bz), ndim=2)
    p = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_GCA, fixed_iters=4, gyro_phase=1)
    x, uo, dxp, fl, det = O.step_one(field, p, np.array([3.0, 3.0]), u.copy(), np.zeros(2))
    assert det.branch == 0 and det.upar_new == pytest.approx(0.0, abs=1e-14)
    assert np.allclose(det.bpg[:], bp, atol=1e-14)
    ug = uo - vE * Gam
    phi = -qm * Bz * dt / (kappa * Gam)
    assert np.allclose(ug, up * rot_z(bp, phi), rtol=0, atol=1e-13)
