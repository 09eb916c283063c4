"""Pins of the oracle's dual-number gradient (oracle/gcb_oracle_grad.cpp), the
reference the adjoint of the CUDA library is compared with.

- Its values are the oracle's: the same initial state pushed by the C oracle
  and by the dual-number code ends in the same final state (bitwise: the two
  follow the same arithmetic in the same order).
- Closed forms in uniform fields on the grid, with one mode whose pattern is
  a uniform electric field of amplitude a:
    E parallel to B: each step adds q dt E/m to the momentum along B on both
    branches (Boris, Sec. 2.1: the rotation about B leaves |u_perp| and u_par
    unchanged; GCA, Sec. 2.2.1: the u_par kick, with |u_perp,g| kept by mu at
    constant B), so Gamma_final = sqrt(1 + |u_perp,0|^2 + (u_par,0 + n q dt a
    E/m)^2) and its derivatives with respect to a and u0 follow;
    E normal to B (GCA): the guiding center drifts with v_E = c E x B/B^2
    (Sec. 2.2), so x_final = x0 + n dt a E/B along E x B.
- Central differences of the C oracle (step h and h/2, compared where they
  agree) on a small case of the differentiation workload, for every final
  state component with respect to every amplitude and initial momentum.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2007_14401_gb300 import inputs
from tests.helpers import copy_state, oracle_field, oracle_params

NX, NY = 16, 8


def uniform_grid(E, B):
    one = np.ones((NY, NX))
    return dict(E=[e * one for e in E], B=[b * one for b in B],
                dB=[0.0 * one for _ in range(6)], dx=(1.0, 1.0))


def state_of(x, u, species=0):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(2, -1))
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3, -1))
    n = x.shape[1]
    return dict(x=x, u=u, dxp=np.zeros((2, n)), flags=np.full(n, species << 6, dtype=np.uint8))


def gamma_rows(st, jac):
    """d Gamma_final / d(a..., u0) from the Jacobian rows of u_final."""
    u = st["u"]
    G = np.sqrt(1.0 + (u * u).sum(0))
    return G, np.einsum("kn,nkj->nj", u / G, jac[:, 2:5, :])


def test_values_equal_the_c_oracle():
    base, pats, amps, st0, p = inputs.reconnection_2d_modes(
        nx=64, ny=32, delta=2.0, n_modes=6, max_mode=2, n_particles=256, omega_dt_max=5.0,
        seed=3)
    for fixed in (4, 0):
        prm = oracle_params(p, gca_fixed_iters=fixed)
        ref = copy_state(st0)
        O.push_sr(ref, oracle_field(inputs.combine_fields(base, pats, amps)), prm, 10)
        got = copy_state(st0)
        O.push_jac(got, base, pats, amps, prm, 10)
        for k in ("x", "u", "dxp", "flags"):
            assert np.array_equal(got[k], ref[k]), (fixed, k)
    # both branches and GCA failures are on the path
    assert 0 < np.mean(ref["flags"] & 1) < 1


@pytest.mark.parametrize("force", [O.FORCE_BORIS, O.FORCE_GCA])
def test_parallel_field_closed_form(force):
    """E = a E_p z-hat, B = B0 z-hat, n steps: u_z gains n q dt a E_p/m, the
    perpendicular momentum keeps its magnitude, in-plane positions stay put
    on the GCA branch (b = z-hat, v_E = 0)."""
    B0, Ep, a, qm, dt, n = 2.0, 0.3, 0.7, -1.5, 0.2, 9
    base = uniform_grid((0, 0, 0), (0, 0, B0))
    pat = uniform_grid((0, 0, Ep), (0, 0, 0))
    u0 = np.array([[0.4, -0.2], [0.3, 0.5], [0.2, -0.6]])
    st = state_of([[3.3, 7.1], [2.2, 5.9]], u0.copy())
    prm = O.make_params(dt=dt, qm=(qm,), grad_mode=O.GRAD_GRID, force=force, fixed_iters=3,
                        f_rho=1e9)
    jac = O.push_jac(st, base, [pat], [a], prm, n)
    uz = u0[2] + n * qm * dt * a * Ep
    uperp2 = u0[0] ** 2 + u0[1] ** 2
    Gf = np.sqrt(1 + uperp2 + uz * uz)
    assert np.allclose(st["u"][2], uz, rtol=1e-14, atol=1e-14)
    assert np.allclose(st["u"][0] ** 2 + st["u"][1] ** 2, uperp2, rtol=1e-13)
    G, dG = gamma_rows(st, jac)
    assert np.allclose(G, Gf, rtol=1e-14)
    want = np.stack([uz * n * qm * dt * Ep / Gf, u0[0] / Gf, u0[1] / Gf, uz / Gf], axis=1)
    assert np.allclose(dG, want, rtol=1e-12, atol=1e-14)
    # u_z's own derivative: d/da = n q dt E_p / m, d/du0_z = 1, d/du0_xy = 0
    assert np.allclose(jac[:, 4, :], [[n * qm * dt * Ep, 0.0, 0.0, 1.0]] * 2, atol=1e-13)
    if force == O.FORCE_GCA:
        assert np.array_equal(st["x"], [[3.3, 7.1], [2.2, 5.9]])
        assert np.all(jac[:, 0:2, :] == 0.0)


def test_exb_drift_closed_form():
    """GCA in E = a E_p y-hat, B = B0 z-hat: v_E = a E_p/B0 x-hat, so after n
    steps dx/da = n dt E_p/B0, dx/du0 = 0, dy/d(.) = 0."""
    B0, Ep, a, qm, dt, n = 1.5, 0.2, 0.5, 2.0, 0.3, 7
    base = uniform_grid((0, 0, 0), (0, 0, B0))
    pat = uniform_grid((0, Ep, 0), (0, 0, 0))
    st = state_of([[1.5, 4.25], [6.5, 2.75]], [[0.1, -0.3], [0.2, 0.1], [0.4, 0.3]], species=1)
    prm = O.make_params(dt=dt, qm=(-qm, qm), grad_mode=O.GRAD_GRID, force=O.FORCE_GCA,
                        fixed_iters=3)
    x0 = st["x"].copy()
    jac = O.push_jac(st, base, [pat], [a], prm, n)
    drift = n * dt * a * Ep / B0
    assert np.allclose(st["x"][0], (x0[0] + drift) % NX, rtol=1e-13)
    assert np.allclose(st["x"][1], x0[1], rtol=1e-14)
    assert np.allclose(jac[:, 0, 0], n * dt * Ep / B0, rtol=1e-12)
    assert np.allclose(jac[:, 0, 1:], 0.0, atol=1e-14)
    assert np.allclose(jac[:, 1, :], 0.0, atol=1e-14)


@pytest.fixture(scope="module")
def fd_case():
    base, pats, amps, st0, p = inputs.reconnection_2d_modes(
        nx=64, ny=32, delta=2.0, n_modes=4, max_mode=2, n_particles=192, omega_dt_max=5.0,
        seed=7)
    prm = oracle_params(p, gca_fixed_iters=4)
    return base, pats, amps, st0, prm


def oracle_final(base, pats, amps, st, prm, n_steps):
    s = copy_state(st)
    O.push_sr(s, oracle_field(inputs.combine_fields(base, pats, amps)), prm, n_steps)
    return s


def final_vec(s, ref, L):
    dx = s["x"] - ref["x"]
    dx -= np.asarray(L)[:, None] * np.round(dx / np.asarray(L)[:, None])
    return np.concatenate([dx, s["u"], s["dxp"]], axis=0)       # (7, n)


def test_jacobian_against_central_differences(fd_case):
    base, pats, amps, st0, prm = fd_case
    n_steps, L = 8, (64.0, 32.0)
    got = copy_state(st0)
    jac = O.push_jac(got, base, pats, amps, prm, n_steps)
    ref = oracle_final(base, pats, amps, st0, prm, n_steps)
    M = len(amps)
    fds = {}
    for h in (1e-6, 5e-7):
        cols = []
        for j in range(M + 3):
            pm = []
            for sgn in (1, -1):
                if j < M:
                    a = amps.copy()
                    a[j] += sgn * h
                    s = oracle_final(base, pats, a, st0, prm, n_steps)
                else:
                    s0 = copy_state(st0)
                    s0["u"][j - M] += sgn * h
                    s = oracle_final(base, pats, amps, s0, prm, n_steps)
                pm.append(final_vec(s, ref, L))
            cols.append((pm[0] - pm[1]) / (2 * h))
        fds[h] = np.stack(cols, axis=2).transpose(1, 0, 2)          # (n, 7, M+3)
    a, b = fds[1e-6], fds[5e-7]
    scale = np.sqrt(np.mean(b ** 2, axis=0, keepdims=True)) + 1e-12
    smooth = np.abs(a - b) <= 1e-5 * (np.abs(b) + scale) + 1e-8
    per_particle = smooth.all(axis=(1, 2))
    assert per_particle.mean() > 0.9
    err = np.abs(jac - b) / (np.abs(b) + scale)
    assert np.all(err[per_particle] < 1e-5), float(err[per_particle].max())
    # the momentum columns of a particle's own u are seeded at 1
    assert np.abs(jac[:, 2:5, M:]).max() > 0.1
