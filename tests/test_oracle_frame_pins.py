"""Pins of the oracle's exact drift frame (Sec. 2.2, Beklemishev & Tessarotto):
the frame moving with v_E sees E and B parallel, with field direction b*.

- Lorentz invariants: B'^2 - E'^2 = B^2 - E^2 and E' B' = E.B.
- An explicit Lorentz transformation of (E, B) into the frame moving with
  v_E gives parallel fields of magnitudes E', B' (signs as E.B), whose
  magnetic direction is b*; b* is a unit vector normal to v_E, and v_E is
  along E x B.
- E.B = 0: b* = b, v_E = c E x B / B^2 (the simplified frame the paper's
  schemes use) to rounding; E parallel to B: b* = b, v_E = 0.
- First order in E.B: u_par b* = u_par b + u_rel with the paper's
  u_rel = u_par (E.B) (b / B'^2) x (E x B) / B^2, B' = B sqrt(1 - E_perp^2/B^2),
  the difference falling as (E.B)^2.
- The guiding-center step in the exact frame (uniform fields, E.B != 0):
  the guiding center moves by dt (u_par b*/Gamma + v_E) with Gamma = kappa
  sqrt(1 + u_par^2 + 2 mu B kappa/m) (Eq. lfacgca2 in that frame), u_par
  gains q dt E.b*/m, and the simplified frame's step is unchanged.
"""
import math

import numpy as np
import pytest

import oracle as O


def boost(E, B, v):
    """Fields in the frame moving with velocity v (c = 1)."""
    v = np.asarray(v, float)
    g = 1.0 / math.sqrt(1.0 - v @ v)
    Ep = g * (E + np.cross(v, B)) - g * g / (g + 1.0) * v * (v @ E)
    Bp = g * (B - np.cross(v, E)) - g * g / (g + 1.0) * v * (v @ B)
    return Ep, Bp


def random_fields(rng, ratio):
    B = rng.standard_normal(3)
    E = rng.standard_normal(3)
    E *= ratio * np.linalg.norm(B) / np.linalg.norm(E)
    return E, B


@pytest.mark.parametrize("ratio", [0.05, 0.5, 0.9, 1.5])
def test_invariants_boost_and_direction(ratio):
    rng = np.random.default_rng(int(ratio * 100))
    for _ in range(20):
        E, B = random_fields(rng, ratio)
        vE, bs, kappa, Ep, Bp = O.bt_frame(E, B)
        assert Bp * Bp - Ep * Ep == pytest.approx(B @ B - E @ E, rel=1e-12, abs=1e-14)
        assert Ep * Bp == pytest.approx(E @ B, rel=1e-12, abs=1e-14)
        assert np.linalg.norm(bs) == pytest.approx(1.0, abs=1e-14)
        assert abs(bs @ vE) <= 1e-14 * (1 + np.linalg.norm(vE))
        ExB = np.cross(E, B)
        assert np.linalg.norm(np.cross(vE, ExB)) <= 1e-13 * np.linalg.norm(ExB) * np.linalg.norm(vE)
        assert kappa == pytest.approx(1.0 / math.sqrt(1.0 - vE @ vE), rel=1e-14)
        Eb, Bb = boost(E, B, vE)
        assert np.linalg.norm(np.cross(Eb, Bb)) <= 1e-12 * np.linalg.norm(Eb) * np.linalg.norm(Bb) + 1e-15
        assert np.linalg.norm(Bb) == pytest.approx(Bp, rel=1e-12)
        assert np.linalg.norm(Eb) == pytest.approx(abs(Ep), rel=1e-11, abs=1e-14)
        assert np.allclose(Bb / np.linalg.norm(Bb), bs, rtol=0, atol=1e-12)


def test_limits():
    rng = np.random.default_rng(3)
    for _ in range(20):
        B = rng.standard_normal(3)
        E = np.cross(rng.standard_normal(3), B)          # E.B = 0
        E *= 0.4 * np.linalg.norm(B) / np.linalg.norm(E)
        vE, bs, kappa, Ep, Bp = O.bt_frame(E, B)
        b = B / np.linalg.norm(B)
        assert np.allclose(bs, b, rtol=0, atol=1e-15)
        assert np.allclose(vE, np.cross(E, B) / (B @ B), rtol=0, atol=1e-15)
        assert abs(Ep) <= 1e-15 * np.linalg.norm(E)           # E.B = 0 up to its rounding
        E = 0.3 * B                                      # E parallel to B
        vE, bs, kappa, Ep, Bp = O.bt_frame(E, B)
        assert np.allclose(bs, b, rtol=0, atol=1e-15)
        assert np.all(np.abs(vE) <= 1e-15) and abs(kappa - 1.0) <= 1e-15


def test_first_order_relativistic_drift():
    """u_par b* - (u_par b + u_rel) = O((E.B)^2): halving E.B quarters it."""
    B = np.array([0.2, -0.1, 1.0])
    Eperp = np.cross(np.array([0.3, 0.7, 0.1]), B)
    Eperp *= 0.3 * np.linalg.norm(B) / np.linalg.norm(Eperp)
    bhat = B / np.linalg.norm(B)
    upar = 1.7
    diffs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        E = Eperp + eps * bhat
        vE, bs, kappa, Ep, Bp = O.bt_frame(E, B)
        EB, B2 = E @ B, B @ B
        Ep2 = Eperp @ Eperp
        Bp2 = B2 * (1.0 - Ep2 / B2)
        urel = upar * EB * np.cross(bhat / Bp2, np.cross(E, B)) / B2
        diffs.append(np.linalg.norm(upar * bs - (upar * bhat + urel)))
        assert np.linalg.norm(urel) > 10 * diffs[-1]
        assert abs(urel @ bhat) <= 1e-15           # u_rel is normal to b
    assert diffs[0] / diffs[1] == pytest.approx(4.0, rel=0.05)
    assert diffs[1] / diffs[2] == pytest.approx(4.0, rel=0.05)


def test_guiding_center_step_in_the_exact_frame():
    """Uniform E, B with E.B != 0, GCA forced, zero curvature terms (uniform
    fields): one step of the exact frame against its closed form, and the
    simplified frame's step left as it was."""
    E = np.array([0.05, 0.12, 0.03])
    B = np.array([0.0, 0.0, 1.0])
    u = np.array([0.4, -0.3, 0.8])
    x = np.array([3.0, 4.0, 0.0])
    dt, qm = 0.45, -20.0
    field = O.uniform_field(E, B, ndim=2)
    kw = dict(dt=dt, qm=(qm,), force=O.FORCE_GCA, fixed_iters=4, curvature=1)
    for frame in (O.FRAME_SIMPLE, O.FRAME_BT):
        p = O.make_params(frame=frame, **kw)
        dxp = np.array([0.0, 0.0, 0.0])
        xo, uo, dxo, fl, det = O.step_one(field, p, x.copy(), u.copy(), dxp)
        if frame == O.FRAME_BT:
            vE, b, kappa, _, _ = O.bt_frame(E, B)
        else:
            vE, b = np.cross(E, B) / (B @ B), B / np.linalg.norm(B)
            kappa = 1.0 / math.sqrt(1.0 - vE @ vE)
        G0 = math.sqrt(1.0 + u @ u)
        upar0 = u @ b
        ug = u - upar0 * b - vE * G0
        mu = (ug @ ug) / (2.0 * kappa)          # mu/m with |B| = 1
        upar1 = upar0 + qm * dt * (E @ b)
        G1 = kappa * math.sqrt(1.0 + upar1 ** 2 + 2.0 * mu * kappa)
        R1 = x[:2] + dt * (upar1 * b / G1 + vE)[:2]
        assert det.branch == 0 and det.iters == 4
        assert det.upar_new == pytest.approx(upar1, rel=1e-13)
        assert np.allclose(xo[:2], R1, rtol=1e-13, atol=1e-14)
        want_u = upar1 * b + vE * G1 + math.sqrt(2.0 * mu * kappa) * ug / np.linalg.norm(ug)
        assert np.allclose(uo, want_u, rtol=1e-12, atol=1e-13)
