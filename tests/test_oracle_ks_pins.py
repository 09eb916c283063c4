"""Pins of the covariant (Kerr-Schild) oracle, CPU only.

Facts used: the Kerr determinant det g = -rho^4 sin^2(theta); the event
horizon r_h = 1 + sqrt(1 - a^2) where g^{rr} = 0; the Minkowski limit;
finite differences of the metric; frame invariants; conservation of u_phi
(axisymmetry) and of E = alpha Gamma - beta^i u_i (stationarity) along
geodesics; Bardeen-Press-Teukolsky circular equatorial orbits; the flat-space
cell area; and the paper's discrete IMR equations of Sec. 2.3 and 2.4.
"""
import math

import numpy as np
import pytest

import oracle as O

A = 0.9


def line_element_4d(a, r, th):
    """g_{mu nu} rebuilt from the oracle's 3+1 quantities."""
    m = O.ks_metric(a, r, th)
    bdn = m["gdn"] @ m["beta"]
    g = np.zeros((4, 4))
    g[0, 0] = -m["alpha"] ** 2 + bdn @ m["beta"]
    g[0, 1:] = g[1:, 0] = bdn
    g[1:, 1:] = m["gdn"]
    return g, m


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9, 0.999])
@pytest.mark.parametrize("r,th", [(1.7, 0.3), (3.0, 1.2), (12.0, math.pi / 2), (40.0, 2.9)])
def test_metric_identities(a, r, th):
    g, m = line_element_4d(a, r, th)
    rho2 = r * r + a * a * math.cos(th) ** 2
    assert np.linalg.det(g) == pytest.approx(-rho2 ** 2 * math.sin(th) ** 2, rel=1e-12)
    assert np.allclose(m["gdn"] @ m["gup"], np.eye(3), atol=1e-12)
    assert m["sqrtg"] ** 2 == pytest.approx(np.linalg.det(m["gdn"]), rel=1e-12)
    gi = np.linalg.inv(g)
    assert gi[0, 0] == pytest.approx(-1.0 / m["alpha"] ** 2, rel=1e-10)
    assert np.allclose(gi[1:, 1:], m["gup"] - np.outer(m["beta"], m["beta"]) / m["alpha"] ** 2,
                       atol=1e-10)


@pytest.mark.parametrize("a", [0.3, 0.9, 0.999])
def test_horizon_where_grr_vanishes(a):
    rh = 1 + math.sqrt(1 - a * a)
    for th in (0.4, 1.3, 2.5):
        m = O.ks_metric(a, rh, th)
        grr = m["gup"][0, 0] - m["beta"][0] ** 2 / m["alpha"] ** 2
        assert abs(grr) < 1e-12
        m2 = O.ks_metric(a, rh * 1.01, th)
        assert m2["gup"][0, 0] - m2["beta"][0] ** 2 / m2["alpha"] ** 2 > 0


def test_minkowski_limit():
    r, th = 1e7, 1.1
    m = O.ks_metric(0.0, r, th)
    assert m["alpha"] == pytest.approx(1.0, abs=1e-6)
    assert abs(m["beta"][0]) < 1e-6
    assert np.allclose(m["gdn"], np.diag([1.0, r * r, (r * math.sin(th)) ** 2]), rtol=1e-6)


@pytest.mark.parametrize("r,th", [(2.1, 0.7), (5.0, 1.5), (20.0, 2.2)])
def test_dual_derivatives_match_differences(r, th):
    m = O.ks_metric(A, r, th)
    for i, h in ((0, 1e-6 * r), (1, 1e-6)):
        xp = [r, th]
        xm = [r, th]
        xp[i] += h
        xm[i] -= h
        p_, q_ = O.ks_metric(A, *xp), O.ks_metric(A, *xm)
        assert m["dalpha"][i] == pytest.approx((p_["alpha"] - q_["alpha"]) / (2 * h), rel=1e-7,
                                               abs=1e-10)
        assert np.allclose(m["dbeta"][i], (p_["beta"] - q_["beta"]) / (2 * h), rtol=1e-7,
                           atol=1e-10)
        assert np.allclose(m["dgup"][i], (p_["gup"] - q_["gup"]) / (2 * h), rtol=1e-6,
                           atol=1e-9)
    assert np.all(m["dalpha"][2] == 0) and np.all(m["dgup"][2] == 0)


def test_local_frame_invariants():
    rng = np.random.default_rng(1)
    for _ in range(10):
        r, th = rng.uniform(1.5, 30), rng.uniform(0.1, 3.0)
        u, F = rng.normal(size=3), rng.normal(size=3)
        m = O.ks_metric(A, r, th)
        uh, Fh = O.ks_frame(A, r, th, u, F)
        assert uh @ uh == pytest.approx(u @ m["gup"] @ u, rel=1e-12)
        assert Fh @ Fh == pytest.approx(F @ m["gdn"] @ F, rel=1e-12)
        assert uh @ Fh == pytest.approx(u @ F, rel=1e-12, abs=1e-12)


def vacuum():
    return O.OracleKsField(O.KS_VACUUM)


def energy(a, x, u):
    m = O.ks_metric(a, x[0], x[1])
    G = math.sqrt(1 + u @ m["gup"] @ u)
    return m["alpha"] * G - m["beta"] @ u


def run_geodesic(a, x, u, dt, n, tol=1e-14):
    f = vacuum()
    kp = O.ks_params(a, 1.0, 1e9)
    p = O.make_params(dt=dt, qm=(-1.0,), force=O.FORCE_BORIS, tol=tol, max_iter=60)
    xs = [np.array(x, float)]
    for _ in range(n):
        x, u, fl, det = O.ks_step_one(f, kp, p, x, u)
        assert det.branch == 1 and not det.nonconv
        xs.append(x.copy())
    return np.array(xs), u


def test_geodesic_conserves_uphi_exactly_and_energy_at_second_order():
    x0 = np.array([8.0, 1.1, 0.3])
    u0 = np.array([-0.1, 0.6, 3.1])
    errs = []
    for dt in (0.2, 0.1):
        n = int(round(40 / dt))
        xs, u = run_geodesic(A, x0, u0, dt, n)
        assert u[2] == pytest.approx(u0[2], rel=1e-13)
        errs.append(abs(energy(A, xs[-1], u) - energy(A, x0, u0)))
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def circular_orbit(a, r):
    """Prograde circular equatorial orbit (Bardeen, Press & Teukolsky 1972):
    specific energy E and angular momentum L; u_r from the Kerr-Schild g_{r mu}."""
    sr = math.sqrt(r)
    den = r ** 0.75 * math.sqrt(r ** 1.5 - 3 * sr + 2 * a)
    E = (r ** 1.5 - 2 * sr + a) / den
    L = (r * r - 2 * a * sr + a * a) / den
    Om = 1.0 / (r ** 1.5 + a)
    z = 2.0 / r
    gtt, gtp, gpp = -(1 - z), -a * z, r * r + a * a + z * a * a
    ut = 1.0 / math.sqrt(-(gtt + 2 * gtp * Om + gpp * Om * Om))
    u_r = ut * (z - a * (1 + z) * Om)          # g_rt u^t + g_rphi u^phi
    return E, L, np.array([u_r, 0.0, L]), Om


def test_circular_equatorial_orbit_stays_circular():
    r0 = 6.0
    E, L, u0, Om = circular_orbit(A, r0)
    x0 = np.array([r0, math.pi / 2, 0.0])
    assert energy(A, x0, u0) == pytest.approx(E, rel=1e-12)
    # the orbit is an equilibrium of the discrete scheme too (G_r = 0 there):
    # r and theta stay put, phi advances at Omega = 1 / (r^{3/2} + a)
    dt = 0.4
    n = int(round(2 * math.pi / Om / dt))
    xs, u = run_geodesic(A, x0, u0, dt, n)
    assert np.max(np.abs(xs[:, 0] - r0)) < 1e-9
    assert np.max(np.abs(xs[:, 1] - math.pi / 2)) < 1e-12
    dphi = np.diff(np.unwrap(xs[:, 2]))
    assert np.allclose(dphi / dt, Om, rtol=1e-9)
    # a slightly eccentric start oscillates about r0 with amplitude ~ the kick
    u1 = u0 + np.array([0.01, 0.0, 0.0])
    xs, u = run_geodesic(A, x0, u1, dt, n)
    assert 0.0 < np.max(np.abs(xs[:, 0] - r0)) < 0.5


def test_cell_sizes_flat_limit_and_quadrature():
    nr, nth = 9, 7
    logr0, dlogr = math.log(1e5), 0.05
    D = [np.zeros((nth, nr))] * 3
    f = O.OracleKsField(O.KS_GRID, nr, nth, logr0, dlogr, D=D, B=D)
    dl = O.ks_cell_sizes(f, 0.0)
    dth = math.pi / (nth - 1)
    for j in range(nth - 1):
        for i in range(nr - 1):
            r0, r1 = math.exp(logr0 + i * dlogr), math.exp(logr0 + (i + 1) * dlogr)
            assert dl[j, i] ** 2 == pytest.approx(0.5 * (r1 * r1 - r0 * r0) * dth, rel=2e-5)
    # near the hole: against an adaptive quadrature of the same element
    from scipy.integrate import dblquad
    f2 = O.OracleKsField(O.KS_GRID, 5, 5, math.log(2.0), 0.1, D=[np.zeros((5, 5))] * 3,
                         B=[np.zeros((5, 5))] * 3)
    dl2 = O.ks_cell_sizes(f2, A)

    def elem(th, r):
        rho2 = r * r + A * A * math.cos(th) ** 2
        return math.sqrt((1 + 2 * r / rho2) * rho2)

    r0, r1 = 2.0 * math.exp(0.1), 2.0 * math.exp(0.2)
    val, _ = dblquad(elem, r0, r1, math.pi / 4, math.pi / 2)
    assert dl2[1, 1] ** 2 == pytest.approx(val, rel=1e-7)


def monopole(B0=50.0, a=0.0):
    return O.OracleKsField(O.KS_MONOPOLE, par=[B0, a])


def test_grgca_step_solves_the_discrete_imr_equations():
    """GRGCA (Sec. 2.4): R^{n+1} - R^n = dt V~(Rb, ub), u'' - u' = dt G(Rb, ub).b(Rb)."""
    a, B0, qm, dt = 0.6, 40.0, -30.0, 0.3
    f = monopole(B0, a)
    kp = O.ks_params(a, 1.0, 1e9)
    p = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_GCA, fixed_iters=60)
    x0 = np.array([7.0, 1.0, 0.2])
    m0 = O.ks_metric(a, *x0[:2])
    Bup = np.array([B0 * math.sin(x0[1]) / m0["sqrtg"], 0, 0])
    Bdn = m0["gdn"] @ Bup
    Bm = math.sqrt(Bdn @ Bup)
    u0 = 0.7 * Bdn / Bm + np.array([0.0, 0.3, 0.5])
    x1, u1, fl, det = O.ks_step_one(f, kp, p, x0, u0)
    assert det.branch == 0 and det.gcafail == 0
    # D = 0: the half kicks vanish, u' = u_par^n and u_par^{n+1} = u''
    up, un, mu = det.upar_old, det.upar_new, det.mu
    Rb = 0.5 * (x0 + x1)
    ub = 0.5 * (up + un)
    m = O.ks_metric(a, Rb[0], Rb[1])
    Bu = np.array([B0 * math.sin(Rb[1]) / m["sqrtg"], 0, 0])
    Bd = m["gdn"] @ Bu
    B = math.sqrt(Bd @ Bu)
    bdn, bup = Bd / B, Bu / B
    Gam = math.sqrt(1 + ub * ub + 2 * mu * B)        # kappa = 1 (no D)
    V = m["alpha"] * (ub * m["gup"] @ bdn / Gam) - m["beta"]
    assert np.allclose(x1 - x0, dt * V, atol=1e-12)
    # u_bar from the reconstruction with the gyration direction held fixed
    ug0 = u0 - up * (m0["gdn"] @ (Bup / Bm))
    n0 = math.sqrt(ug0 @ m0["gup"] @ ug0)
    ubar = ub * bdn + math.sqrt(2 * mu * B) * ug0 / n0
    G = np.array([-Gam * m["dalpha"][i] + ubar @ m["dbeta"][i]
                  - m["alpha"] * ubar @ m["dgup"][i] @ ubar / (2 * Gam) for i in range(3)])
    assert un - up == pytest.approx(dt * G @ bup, abs=1e-12)


def test_grgca_flat_limit_drift_is_the_special_relativistic_one():
    """Far from a non-spinning hole, in the local frame the guiding center moves
    at u_par b/Gamma + D x B / B^2 (Sec. 2.4 reduces to Sec. 2.2.1)."""
    a, r = 0.0, 1e6
    nr, nth = 4, 181
    logr0, dlogr = math.log(r) - 1e-3, 1e-3
    th_nodes = np.linspace(0, math.pi, nth)
    # uniform local-frame fields near theta = pi/2: B^ along r^, D^ along th^
    Bh, Dh = 2.0, 0.3
    D = [np.zeros((nth, nr)), np.zeros((nth, nr)), np.zeros((nth, nr))]
    B = [np.zeros((nth, nr)), np.zeros((nth, nr)), np.zeros((nth, nr))]
    for j, th in enumerate(th_nodes):
        for i in range(nr):
            rr = math.exp(logr0 + i * dlogr)
            m = O.ks_metric(a, rr, th)
            B[0][j, i] = Bh / math.sqrt(m["gdn"][0, 0])
            D[1][j, i] = Dh / math.sqrt(m["gdn"][1, 1])
    f = O.OracleKsField(O.KS_GRID, nr, nth, logr0, dlogr, D=D, B=B)
    kp = O.ks_params(a, 1.0, 1e9)
    dt = 0.5
    p = O.make_params(dt=dt, qm=(-1000.0,), force=O.FORCE_GCA, fixed_iters=30)
    x0 = np.array([r * math.exp(5e-4), math.pi / 2 + 1e-4, 0.0])
    m = O.ks_metric(a, *x0[:2])
    upar = 0.4
    vE = Dh / Bh                                 # |D^ x B^| / B^2, along -phi^ here
    kappa = 1 / math.sqrt(1 - vE * vE)
    G0 = kappa * math.sqrt(1 + upar * upar)      # no gyration: u = u_par b + v_E Gamma
    u0 = np.array([upar * math.sqrt(m["gdn"][0, 0]), 0.0, -vE * G0 * math.sqrt(m["gdn"][2, 2])])
    x1, u1, fl, det = O.ks_step_one(f, kp, p, x0, u0)
    assert det.branch == 0
    assert det.mu == pytest.approx(0.0, abs=1e-12)
    Gam = kappa * math.sqrt(1 + det.upar_new ** 2)
    # coordinate displacement -> local-frame (orthonormal) components
    dr = (x1[0] - x0[0]) * math.sqrt(m["gdn"][0, 0]) / dt
    dphi = (x1[2] - x0[2] + math.pi) % (2 * math.pi) - math.pi
    dph = dphi * math.sqrt(m["gdn"][2, 2]) / dt
    assert dr == pytest.approx(det.upar_new / Gam, rel=1e-4)
    assert dph == pytest.approx(-vE, rel=1e-4)      # D^ x B^ points along -phi^ here
    # D . b = 0: only the geodesic term of spherical coordinates, ~ v_E^2 dt / r
    assert det.upar_new == pytest.approx(upar, abs=1e-7)


def test_greom_half_kicks_rotate_in_the_local_frame():
    """Far from a non-spinning hole with a uniform local field B^ = B r^, the two
    half kicks of a GREOM step (Sec. 2.3, Boris over alpha dt / 2 each) keep
    |u^| and turn u^ about r^ by 4 atan(|q/m| alpha dt B / (4 gamma))."""
    a, r, Bh, qm, dt = 0.0, 1e6, 3.0, -2.0, 0.4
    nr, nth = 4, 181
    logr0, dlogr = math.log(r) - 1e-3, 1e-3
    th_nodes = np.linspace(0, math.pi, nth)
    Z = [np.zeros((nth, nr)) for _ in range(3)]
    B = [np.zeros((nth, nr)), np.zeros((nth, nr)), np.zeros((nth, nr))]
    for j, th in enumerate(th_nodes):
        for i in range(nr):
            m = O.ks_metric(a, math.exp(logr0 + i * dlogr), th)
            B[0][j, i] = Bh / math.sqrt(m["gdn"][0, 0])
    f = O.OracleKsField(O.KS_GRID, nr, nth, logr0, dlogr, D=Z, B=B)
    kp = O.ks_params(a, 1.0, 1e9)
    p = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_BORIS, tol=1e-15, max_iter=50)
    x0 = np.array([r * math.exp(5e-4), math.pi / 2, 1.0])
    m = O.ks_metric(a, *x0[:2])
    uh0 = np.array([0.0, 0.3, 0.4])                       # perpendicular to r^
    u0 = uh0 * np.sqrt(np.diag(m["gdn"]))
    x1, u1, fl, det = O.ks_step_one(f, kp, p, x0, u0)
    m1 = O.ks_metric(a, *x1[:2])
    uh1 = u1 / np.sqrt(np.diag(m1["gdn"]))
    g = math.sqrt(1 + uh0 @ uh0)
    ang = 4 * math.atan(abs(qm) * m["alpha"] * dt * Bh / (4 * g))
    assert np.linalg.norm(uh1) == pytest.approx(np.linalg.norm(uh0), rel=1e-9)
    got = math.atan2(uh0[1] * uh1[2] - uh0[2] * uh1[1], uh0[1] * uh1[1] + uh0[2] * uh1[2])
    assert abs(got) == pytest.approx(ang, rel=1e-5)
    assert math.copysign(1, got) == -math.copysign(1, qm)   # right-handed about r^ for q < 0


# ---------------------------------------------------------------------------
# The GREOM kick in the global coordinate basis (the option of Sec. 2.3 and
# Sec. 2.4: a Boris-like push without tetrads)
# ---------------------------------------------------------------------------
KICK_POINTS = [(0.9, 1.3, 0.4), (0.9, 1.5, 0.3), (0.9, 3.0, math.pi / 2), (0.5, 40.0, 2.9),
               (0.999, 1.2, 0.01), (0.0, 7.0, 1.0)]


@pytest.mark.parametrize("a,r,th", KICK_POINTS)
def test_global_kick_without_electric_field_is_the_boris_rotation(a, r, th):
    """D = 0: the kick turns u about B, so gamma^{ij} u_i u_j and u_i B^i are
    kept; the part of u normal to B turns by 2 atan(|t|), |t| = |h| |B| / Gamma
    with |B|^2 = gamma_ij B^i B^j and h = (q/m) dtau / 2 (Boris 1970); the turn
    is left-handed about B for q > 0 and right-handed for q < 0."""
    rng = np.random.default_rng(int(r * 1000) + int(th * 100))
    m = O.ks_metric(a, r, th)
    gup, gdn = m["gup"], m["gdn"]
    for qm in (-7.0, 3.0):
        B = rng.normal(size=3) * 2.0
        u = rng.normal(size=3) * 3.0
        dtau = 0.2
        u1 = O.ks_kick(a, r, th, np.zeros(3), B, qm, dtau, u, basis=O.KICK_GLOBAL)
        uu = u @ gup @ u
        assert u1 @ gup @ u1 == pytest.approx(uu, rel=1e-13)
        assert u1 @ B == pytest.approx(u @ B, rel=1e-12, abs=1e-12 * math.sqrt(uu))
        Bn = math.sqrt(B @ gdn @ B)
        b_dn, b_up = gdn @ B / Bn, B / Bn
        p0 = u - (u @ b_up) * b_dn
        p1 = u1 - (u1 @ b_up) * b_dn
        p0u, p1u = gup @ p0, gup @ p1
        cos = p0 @ p1u / (p0 @ p0u)
        sin = m["sqrtg"] * (b_up @ np.cross(p0u, p1u)) / (p0 @ p0u)
        turn = math.atan2(sin, cos)
        h = 0.5 * qm * dtau
        assert abs(turn) == pytest.approx(2 * math.atan(abs(h) * Bn / math.sqrt(1 + uu)), rel=1e-11)
        assert math.copysign(1.0, turn) == -math.copysign(1.0, qm)


@pytest.mark.parametrize("a,r,th", KICK_POINTS)
def test_global_kick_without_magnetic_field_is_linear(a, r, th):
    """B = 0: covariant u_i gains (q/m) dtau gamma_ij D^j exactly."""
    rng = np.random.default_rng(7)
    m = O.ks_metric(a, r, th)
    D, u = rng.normal(size=3), rng.normal(size=3) * 2.0
    qm, dtau = -4.0, 0.3
    u1 = O.ks_kick(a, r, th, D, np.zeros(3), qm, dtau, u, basis=O.KICK_GLOBAL)
    want = u + qm * dtau * (m["gdn"] @ D)
    np.testing.assert_allclose(u1, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())


def test_global_kick_equals_the_local_frame_kick():
    """The frame cross product of L^{-1} a and L^{-1} b maps back to
    sqrt(gamma) [ijk] a^j b^k because det L = 1 / sqrt(gamma), and frame dot
    products are metric contractions: the two bases give one kick."""
    rng = np.random.default_rng(3)
    for a, r, th in KICK_POINTS:
        for scale in (1e-3, 1.0, 1e3):
            D, B = rng.normal(size=3) * 0.3, rng.normal(size=3) * scale
            u = rng.normal(size=3) * rng.choice([0.1, 10.0, 1e3])
            qm, dtau = rng.choice([-1e3, -2.0, 5.0]), 0.05
            uf = O.ks_kick(a, r, th, D, B, qm, dtau, u, basis=O.KICK_TETRAD)
            ug = O.ks_kick(a, r, th, D, B, qm, dtau, u, basis=O.KICK_GLOBAL)
            assert np.abs(ug - uf).max() <= 1e-13 * np.abs(uf).max()


def test_greom_steps_in_both_bases_agree():
    """Whole GREOM steps (half kick, implicit midpoint, half kick) in the Wald
    field, in the local frame and in the global basis: equal up to rounding."""
    from paper_2007_14401_gb300 import inputs
    fields, st, p = inputs.kerr_wald(nr=48, nth=40, n_particles=64, seed=9)
    of = O.ks_grid_field(fields)
    dl = O.ks_cell_sizes(of, p["a"])
    op = O.make_params(dt=p["dt"], f_rho=p["f_rho"], f_E=p["f_E"], qm=(-30.0,),
                       force=O.FORCE_BORIS, fixed_iters=8)
    out = []
    for basis in (O.KICK_TETRAD, O.KICK_GLOBAL):
        s = {k: v.copy() for k, v in st.items()}
        O.push_ks(s, of, O.ks_params(p["a"], p["r_in"], p["r_out"], basis), op, 5, dl=dl)
        out.append(s)
    f, g = out
    live = (f["flags"] & (O.FLAG_EXITED | O.FLAG_NONFINITE)) == 0
    assert live.mean() > 0.9
    np.testing.assert_array_equal(f["flags"], g["flags"])
    dx = np.abs(f["x"] - g["x"])[:, live]
    dx[2] = np.minimum(dx[2], 2 * np.pi - dx[2])
    assert dx.max() <= 1e-12 * np.abs(f["x"][:, live]).max()
    assert np.abs(f["u"] - g["u"])[:, live].max() <= 1e-12 * (np.abs(f["u"][:, live]).max() + 1)


# ---------------------------------------------------------------------------
# The ambient-region test of Sec. 4.2: electrons at rest at r = 5.5 r_g on the
# equator of the Wald field, integrated to t = 20 r_g/c with f_rho = f_E = 1
# and dt = 2 pi / 60 (the step that resolves the gyration at Omega_C0 = c/r_g)
# ---------------------------------------------------------------------------
AMBIENT_T = 20.0
AMBIENT_DT = 2 * math.pi / 60


@pytest.fixture(scope="module")
def ambient():
    from paper_2007_14401_gb300 import inputs
    fields, _, p = inputs.kerr_wald(nr=256, nth=256, Qm=0.0, n_particles=1, seed=0)
    of = O.ks_grid_field(fields)
    dl = O.ks_cell_sizes(of, p["a"])
    kp = O.ks_params(p["a"], p["r_in"], p["r_out"])
    x0 = np.array([5.5, math.pi / 2, 0.0])
    D, B = O.ks_gather(of, x0[0], x0[1])
    m = O.ks_metric(p["a"], x0[0], x0[1])
    Bn = math.sqrt(B @ m["gdn"] @ B)
    return of, dl, kp, x0, Bn


def ambient_run(amb, omega, dt, force, per_step=False):
    """One electron with Omega_C0 = |q/m| B(x0) = omega (rho_C0 = r_g / omega)."""
    of, dl, kp, x0, Bn = amb
    n = int(round(AMBIENT_T / dt))
    st = dict(x=x0[:, None].copy(), u=np.zeros((3, 1)), dxp=np.zeros((3, 1)),
              flags=np.zeros(1, np.uint8))
    op = O.make_params(dt=AMBIENT_T / n, f_rho=1.0, f_E=1.0, qm=(-omega / Bn,), force=force)
    S = []
    if per_step:
        for _ in range(n):
            O.push_ks(st, of, kp, op, 1, dl=dl)
            S.append(int(st["flags"][0] & O.FLAG_S))
    else:
        O.push_ks(st, of, kp, op, n, dl=dl)
    return st["x"][:, 0], np.array(S)


def proper_distance(x, y):
    return math.hypot(x[0] - y[0], y[0] * (x[1] - y[1]), y[0] * (x[2] - y[2]))


@pytest.mark.parametrize("omega", [100.0, 1000.0])
def test_ambient_region_coupled_pusher_tracks_the_resolved_orbit(ambient, omega):
    """Sec. 4.2, ambient region: with rho_C0 <= 1e-2 r_g the sub-grid
    gyration trips the f_rho test, so the coupled pusher takes GRGCA at every
    step, and its trajectory stays on the gyro-resolved GREOM reference
    (dt = 2 pi / (60 Omega_C0)) to within a couple of rho_C0, while plain
    Boris at the coupled pusher's step drifts off by orders of magnitude more."""
    x_c, S = ambient_run(ambient, omega, AMBIENT_DT, O.FORCE_NONE, per_step=True)
    assert len(S) == 191 and not S.any()
    x_ref, _ = ambient_run(ambient, omega, 2 * math.pi / (60 * omega), O.FORCE_BORIS)
    x_b, _ = ambient_run(ambient, omega, AMBIENT_DT, O.FORCE_BORIS)
    d_c, d_b = proper_distance(x_c, x_ref), proper_distance(x_b, x_ref)
    assert d_c < 2.0 / omega, (d_c, 1 / omega)
    assert d_b > 30 * d_c


def test_ambient_region_resolved_gyration_stays_on_boris(ambient):
    """rho_C0 = 1e-1 r_g: the gyro-radius exceeds the cell, the coupled
    pusher never leaves Boris (so it is the Boris pusher) and stays on the
    resolved reference to within the gyro-radius."""
    x_c, S = ambient_run(ambient, 10.0, AMBIENT_DT, O.FORCE_NONE, per_step=True)
    assert S.all()
    x_b, _ = ambient_run(ambient, 10.0, AMBIENT_DT, O.FORCE_BORIS)
    np.testing.assert_array_equal(x_c, x_b)
    x_ref, _ = ambient_run(ambient, 10.0, 2 * math.pi / 600, O.FORCE_BORIS)
    assert proper_distance(x_c, x_ref) < 0.1
