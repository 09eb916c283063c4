"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed
form, an invariant, a brute-force evaluation, an independent derivation
(Lorentz boosts, finite differences) or the residual of the paper's own
discrete equations.  Together they are meant to fail on a dropped term, a
wrong sign, a transposed index or a misplaced factor of c anywhere in the
oracle.  CPU only.
"""
import math

import numpy as np
import pytest

import oracle as O


def unit(v):
    v = np.asarray(v, dtype=float)
    return v / np.linalg.norm(v)


def gamma_of(u, c=1.0):
    return math.sqrt(1.0 + float(np.dot(u, u)) / (c * c))


# --------------------------------------------------------------------------
# L0: linear-shape-function gather (Sec. 4 intro)
# --------------------------------------------------------------------------
def brute_gather(F, dx, x):
    """sum_N F_N W(x - x_N) over every node and periodic image (brute force)."""
    shape = F.shape
    nd = F.ndim
    n = shape[::-1]
    tot = 0.0
    for idx in np.ndindex(*shape):
        ijk = idx[::-1]
        for img in np.ndindex(*([4] * nd)):
            W = 1.0
            for d in range(nd):
                pos = (ijk[d] + (img[d] - 1) * n[d]) * dx[d]
                W *= max(0.0, 1.0 - abs(x[d] - pos) / dx[d])
                if W == 0.0:
                    break
            if W:
                tot += F[idx] * W
    return tot


@pytest.mark.parametrize("ndim", [2, 3])
def test_gather_matches_brute_force(ndim):
    rng = np.random.default_rng(5)
    shape = (3, 4, 5)[-ndim:] if ndim == 3 else (4, 5)
    dx = (0.7, 1.3, 0.9)[:ndim]
    E = [rng.normal(size=shape) for _ in range(3)]
    B = [rng.normal(size=shape) for _ in range(3)]
    f = O.grid_field(E, B, dx)
    p = O.make_params(dt=0.1)
    L = np.array(shape[::-1]) * np.array(dx)
    for _ in range(6):
        x = rng.uniform(-0.5, 1.5, size=ndim) * L
        got = O.eval_field(f, p, x)
        for c in range(3):
            assert got[c] == pytest.approx(brute_gather(E[c], dx, x), abs=1e-12)
            assert got[3 + c] == pytest.approx(brute_gather(B[c], dx, x), abs=1e-12)


@pytest.mark.parametrize("ndim", [2, 3])
def test_gather_gradient_is_derivative_of_interpolant(ndim):
    """grad F = sum F_N grad W: central differences of the brute-force sum
    inside a cell (where the interpolant is multilinear) give it exactly."""
    rng = np.random.default_rng(6)
    shape = (3, 4, 5) if ndim == 3 else (4, 5)
    dx = (0.7, 1.3, 0.9)[:ndim]
    E = [np.zeros(shape) for _ in range(3)]
    B = [rng.normal(size=shape) for _ in range(3)]
    f = O.grid_field(E, B, dx)
    p = O.make_params(dt=0.1, grad_mode=O.GRAD_DW)
    h = 1e-6
    for _ in range(4):
        cell = rng.integers(0, 3, size=ndim)
        frac = rng.uniform(0.1, 0.9, size=ndim)
        x = (cell + frac) * np.array(dx)
        got = O.eval_field(f, p, x)
        for i in range(ndim):
            e = np.zeros(ndim)
            e[i] = h
            for j in range(3):
                fd = (brute_gather(B[j], dx, x + e) - brute_gather(B[j], dx, x - e)) / (2 * h)
                assert got[6 + 3 * i + j] == pytest.approx(fd, abs=1e-7)
        for i in range(ndim, 3):
            assert np.all(got[6 + 3 * i: 9 + 3 * i] == 0.0)


def test_gather_reproduces_linear_field_and_gradient_grid():
    """CIC reproduces a linear field exactly; GRID mode interpolates the given
    gradient grids (constant grids come back unchanged)."""
    nx, ny = 16, 12
    dx = (0.5, 0.25)
    X = np.arange(nx)[None, :] * dx[0] * np.ones((ny, 1))
    Y = np.arange(ny)[:, None] * dx[1] * np.ones((1, nx))
    a, gx, gy = 0.3, -0.7, 1.9
    E = [a + gx * X + gy * Y, np.zeros_like(X), np.ones_like(X)]
    B = [2 * X - Y, 0.5 + Y, -X]
    dB = [np.full_like(X, v) for v in (1.0, 2.0, 3.0, 4.0, 5.0, 6.0)]
    f = O.grid_field(E, B, dx, dB=dB)
    for gm in (O.GRAD_DW, O.GRAD_GRID):
        p = O.make_params(dt=0.1, grad_mode=gm)
        for x in ([1.3, 0.9], [6.1, 2.2], [0.01, 0.02]):
            got = O.eval_field(f, p, x)
            assert got[0] == pytest.approx(a + gx * x[0] + gy * x[1], abs=1e-13)
            assert got[3] == pytest.approx(2 * x[0] - x[1], abs=1e-13)
            assert got[4] == pytest.approx(0.5 + x[1], abs=1e-13)
            assert got[5] == pytest.approx(-x[0], abs=1e-13)
            if gm == O.GRAD_DW:
                want = [2.0, 0.0, -1.0, -1.0, 1.0, 0.0]  # d_x B, d_y B
            else:
                want = [1.0, 2.0, 3.0, 4.0, 5.0, 6.0]
            assert got[6:12] == pytest.approx(want, abs=1e-12)


def test_gather_is_periodic():
    rng = np.random.default_rng(7)
    E = [rng.normal(size=(6, 8)) for _ in range(3)]
    B = [rng.normal(size=(6, 8)) for _ in range(3)]
    f = O.grid_field(E, B, (1.0, 1.0))
    p = O.make_params(dt=0.1)
    for x in ([0.3, 0.4], [7.9, 5.9], [3.5, 2.5]):
        a = O.eval_field(f, p, x)
        b = O.eval_field(f, p, [x[0] + 8.0, x[1] - 6.0])
        assert np.allclose(a, b, atol=1e-13, rtol=0)


# --------------------------------------------------------------------------
# Switch S (Sec. 3, Sec. 4.1)
# --------------------------------------------------------------------------
def test_switch_cases():
    p = O.make_params(dt=0.1, f_rho=0.4, f_E=1.0, dl=1.0)
    # rho~ = 1*1/(1*5) = 0.2 < 0.4, E/B = 0.6 < 1  -> GCA
    S, m = O.switch([3, 0, 0], [0, 5, 0], 1.0, 1.0, p)
    assert S == 0 and m == pytest.approx(min(1 - 0.2 / 0.4, 1 - 0.6))
    # rho~ exactly at the threshold: strict inequality -> Boris
    S, m = O.switch([0, 0, 0], [2.5, 0, 0], 1.0, 1.0, p)
    assert S == 1 and abs(m) < 1e-15
    # E/B exactly f_E -> Boris
    S, _ = O.switch([0, 0, 2], [2, 0, 0], 1.0, 100.0, p)
    assert S == 1
    # B = 0 -> Boris
    S, m = O.switch([0, 0, 0], [0, 0, 0], 1.0, 1.0, p)
    assert S == 1 and m == -math.inf
    # large Gamma gives a large gyro-radius -> Boris
    S, m = O.switch([0, 0, 0], [0, 0, 1], 3.0, 1.0, p)
    assert S == 1 and m < 0
    # f_rho scales the threshold linearly
    p2 = O.make_params(dt=0.1, f_rho=4.0, f_E=1.0, dl=1.0)
    S, _ = O.switch([0, 0, 0], [0, 0, 1], 3.0, 1.0, p2)
    assert S == 0


def test_switch_speed_of_light_scaling():
    """The criterion compares two lengths: under c -> 2c, E -> 2E, B -> 2B,
    dl -> 2 dl (Gamma and q/m fixed) S and its margin are unchanged."""
    rng = np.random.default_rng(8)
    for _ in range(200):
        E = rng.normal(size=3) * 0.3
        B = rng.normal(size=3)
        G = 1.0 + abs(rng.normal()) * 2
        Q = 10 ** rng.uniform(-0.5, 1.5)
        res = []
        for s in (1.0, 2.0):
            p = O.make_params(c=s, dt=0.1, f_rho=0.4, f_E=1.0, dl=s * 1.0)
            res.append(O.switch(s * E, s * B, G, Q, p))
        assert res[0][0] == res[1][0]
        assert res[0][1] == pytest.approx(res[1][1], rel=1e-14, abs=1e-15)


# --------------------------------------------------------------------------
# Boris (Sec. 2.1, standard scheme): closed forms in uniform fields
# --------------------------------------------------------------------------
def rotate(v, axis, ang):
    k = unit(axis)
    return (v * math.cos(ang) + np.cross(k, v) * math.sin(ang)
            + k * np.dot(k, v) * (1 - math.cos(ang)))


@pytest.mark.parametrize("qm", [-2.5, 0.8])
def test_boris_uniform_B_exact_rotation(qm):
    """E = 0: each step rotates u about b by -sgn(q) 2 atan(|q| dt B/(2 m c gamma))
    and moves x by dt u^{n+1/2}/gamma; positions lie on a circle."""
    c = 1.3
    B = np.array([0.3, -0.4, 1.2])
    f = O.uniform_field([0, 0, 0], B)
    p = O.make_params(c=c, dt=0.7, qm=(qm,), force=O.FORCE_BORIS)
    u0 = np.array([0.9, 0.2, -0.5])
    g = gamma_of(u0, c)
    theta = 2 * math.atan(abs(qm) * p.dt * np.linalg.norm(B) / (2 * c * g))
    x, u, dxp = np.zeros(3), u0.copy(), np.zeros(3)
    pts = [x.copy()]
    for _ in range(20):
        x2, u2, dxp2, fl, det = O.step_one(f, p, x, u, dxp, 0)
        want = rotate(u, B, -math.copysign(theta, qm))
        assert np.allclose(u2, want, atol=1e-14 * np.linalg.norm(u0), rtol=0)
        assert np.allclose(dxp2, p.dt * u2 / g, atol=1e-14, rtol=0)
        assert det.branch == 1
        x, u, dxp = x2, u2, dxp2
        pts.append(x.copy())
    b = unit(B)
    uperp = np.linalg.norm(u0 - np.dot(u0, b) * b)
    r_want = p.dt * uperp / (2 * g * math.sin(theta / 2))
    P = [q - np.dot(q, b) * b for q in pts]
    for i in range(len(P) - 2):
        a_, b_, c_ = (np.linalg.norm(P[i + 1] - P[i]), np.linalg.norm(P[i + 2] - P[i + 1]),
                      np.linalg.norm(P[i + 2] - P[i]))
        area = 0.5 * np.linalg.norm(np.cross(P[i + 1] - P[i], P[i + 2] - P[i]))
        assert a_ * b_ * c_ / (4 * area) == pytest.approx(r_want, rel=1e-11)


def test_boris_parallel_E_grows_linearly():
    E0, qm, dt = 0.2, -1.7, 0.3
    B = np.array([0.0, 0.6, 0.8])
    b = unit(B)
    f = O.uniform_field(E0 * b, B)
    p = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_BORIS)
    x, u, dxp = np.zeros(3), np.array([0.4, -0.3, 0.1]), np.zeros(3)
    u0par = np.dot(u, b)
    for n in range(1, 51):
        x, u, dxp, _, _ = O.step_one(f, p, x, u, dxp, 0)
        assert np.dot(u, b) == pytest.approx(u0par + n * qm * E0 * dt, rel=1e-13, abs=1e-13)


def test_boris_energy_conserved_E0_nonuniform():
    """E = 0: the Boris rotation conserves |u| to rounding in any B."""
    f = O.bottle_field(1.0, 3.0)
    p = O.make_params(dt=0.05, qm=(5.0,), force=O.FORCE_BORIS)
    x, u, dxp = np.array([0.3, -0.2, 0.5]), np.array([0.3, 0.5, 0.7]), np.zeros(3)
    n0 = np.linalg.norm(u)
    for _ in range(2000):
        x, u, dxp, _, _ = O.step_one(f, p, x, u, dxp, 0)
    assert np.linalg.norm(u) == pytest.approx(n0, rel=1e-13)


def test_boris_mirrors_in_bottle():
    """Resolved Boris in a magnetic bottle: u_par reverses near the mirror
    point z_m where B(z_m) = B0 |u|^2 / u_perp0^2 (mu invariance)."""
    B0, L = 1.0, 4.0
    f = O.bottle_field(B0, L)
    qm = 50.0
    p = O.make_params(dt=0.002, qm=(qm,), force=O.FORCE_BORIS)
    pitch = math.radians(50.0)
    umag = 0.5
    u = np.array([umag * math.sin(pitch), 0.0, umag * math.cos(pitch)])
    x = np.array([umag * math.sin(pitch) / (qm * B0) * gamma_of(u), 0.0, 0.0])
    dxp = np.zeros(3)
    zmax, flipped = 0.0, False
    for _ in range(30000):
        x, u, dxp, _, _ = O.step_one(f, p, x, u, dxp, 0)
        zmax = max(zmax, x[2])
        if u[2] < 0:
            flipped = True
            break
    zm = L * math.sqrt(1.0 / math.sin(pitch) ** 2 - 1.0)
    assert flipped
    assert zmax == pytest.approx(zm, rel=0.03)


# --------------------------------------------------------------------------
# GCA (Sec. 2.2) against special relativity in uniform fields
# --------------------------------------------------------------------------
def boost(u4, v):
    """Lorentz boost of the 4-vector (Gamma c, u) into the lab, where the
    primed frame moves with velocity v (c = 1)."""
    v = np.asarray(v, float)
    beta = np.linalg.norm(v)
    k = 1.0 / math.sqrt(1 - beta * beta)
    n = v / beta
    L = np.eye(4)
    L[0, 0] = k
    L[0, 1:] = L[1:, 0] = k * v
    L[1:, 1:] += (k - 1) * np.outer(n, n)
    return L @ u4


@pytest.mark.parametrize("upar_p,uperp_p", [(0.7, 0.3), (-1.5, 0.05), (0.0, 0.8)])
def test_gca_uniform_ExB_matches_boosted_gyration(upar_p, uperp_p):
    """Uniform E perp B (E < B): a particle gyrating in the frame drifting at
    v_E = c ExB/B^2 has a guiding center moving at v_E + u_par'/(kappa Gamma') b
    in the lab (boost of the drift-frame motion).  The GCA step must give this
    displacement and leave the (boosted) momentum unchanged."""
    B = np.array([0.0, 0.0, 2.0])
    E = np.array([0.6, 0.0, 0.0])
    vE = np.cross(E, B) / np.dot(B, B)
    kappa = 1 / math.sqrt(1 - np.dot(vE, vE))
    b = unit(B)
    chat = unit(np.cross(b, vE))          # gyration direction perp to v_E and b
    up = upar_p * b + uperp_p * chat
    Gp = gamma_of(up)
    u4 = boost(np.concatenate([[Gp], up]), vE)
    u_lab = u4[1:]
    f = O.uniform_field(E, B)
    p = O.make_params(dt=0.4, qm=(-20.0,), force=O.FORCE_GCA, curvature=1)
    x, u2, dxp, fl, det = O.step_one(f, p, np.array([0.1, 0.2, 0.3]), u_lab, np.zeros(3), 0)
    assert det.branch == 0
    V = vE + upar_p / (kappa * Gp) * b
    assert np.allclose(dxp, p.dt * V, atol=1e-14, rtol=0)
    assert np.allclose(u2, u_lab, atol=1e-13, rtol=0)
    assert det.upar_new == pytest.approx(upar_p, abs=1e-14)


@pytest.mark.parametrize("curv", [0, 1])
def test_gca_parallel_E_second_order(curv):
    """E parallel to B: u_par grows by q E dt/m exactly and the position
    converges at second order to z(t) = (Gamma(t) - Gamma(0)) m c / (q E)."""
    E0, qm, u0, T = 0.05, 1.0, 0.3, 8.0

    def run(dt):
        f = O.uniform_field([0, 0, E0], [0, 0, 1.0])
        p = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_GCA, curvature=curv,
                          fixed_iters=3)
        x, u, dxp = np.zeros(3), np.array([0, 0, u0]), np.zeros(3)
        n = int(round(T / dt))
        for k in range(n):
            x, u, dxp, _, det = O.step_one(f, p, x, u, dxp, 0)
            assert det.upar_new == pytest.approx(u0 + (k + 1) * qm * E0 * dt, abs=1e-13)
        a = qm * E0
        exact = (math.hypot(1, u0 + a * (T + dt / 2)) - math.hypot(1, u0 + a * dt / 2)) / a
        return abs(x[2] - exact)

    e1, e2 = run(0.4), run(0.2)
    assert e1 < 1e-3
    assert 3.5 < e1 / e2 < 4.5


# --------------------------------------------------------------------------
# GCA with curvature: residuals of the paper's discrete equations, with the
# gradients of b taken by finite differences (independent of the oracle's
# analytic d_i b_j).
# --------------------------------------------------------------------------
def frame_fd(f, p, R, h=1e-5):
    F = O.eval_field(f, p, R)
    E, B = F[0:3], F[3:6]
    Bm = np.linalg.norm(B)
    b = B / Bm
    vE = p.c * np.cross(E, B) / Bm ** 2
    kappa = 1 / math.sqrt(1 - np.dot(vE, vE) / p.c ** 2)

    def bdir(d):
        e = np.zeros(3)
        e[: len(R)] = d[: len(R)]
        Fp = O.eval_field(f, p, np.asarray(R) + h * e[: len(R)])
        Fm = O.eval_field(f, p, np.asarray(R) - h * e[: len(R)])
        return (unit(Fp[3:6]) - unit(Fm[3:6])) / (2 * h)

    bgb = bdir(b)
    vgb = bdir(vE)
    return dict(E=E, B=B, Bm=Bm, b=b, vE=vE, kappa=kappa, bgb=bgb, vgb=vgb)


def Gam(fr, upar, mu, c=1.0):
    return fr["kappa"] * math.sqrt(1 + (upar ** 2 + 2 * mu * fr["Bm"] * fr["kappa"]) / c ** 2)


def vcurv(fr, qm, upar, G, c=1.0):
    return (c * fr["kappa"] ** 2 / (qm * fr["Bm"])) * np.cross(
        fr["b"], upar ** 2 / G * fr["bgb"] + upar * fr["vgb"])


def Vgc(fr, qm, upar, mu, c=1.0):
    G = Gam(fr, upar, mu, c)
    return upar * fr["b"] / G + fr["vE"] + vcurv(fr, qm, upar, G, c)


@pytest.mark.parametrize("qm,dt", [(2.0, 0.5), (-30.0, 1.5), (5.0, 4.0)])
def test_gca_curvature_step_solves_discrete_equations(qm, dt):
    f = O.rotor_field(1.0, 0.3, 0.4)
    p = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_GCA, curvature=1, fixed_iters=60)
    Rn = np.array([0.7, 0.2, 0.1])
    fr0 = frame_fd(f, p, Rn)
    assert abs(np.dot(fr0["vE"], fr0["bgb"])) > 1e-3   # curvature terms are active
    assert abs(np.dot(fr0["vE"], fr0["vgb"])) > 1e-3
    u = 0.8 * fr0["b"] + 0.3 * unit(np.cross(fr0["b"], [0.3, 1.0, -0.2])) + 0.2 * fr0["vE"]
    x2, u2, dxp, fl, det = O.step_one(f, p, Rn, u, np.zeros(3), 0)
    assert det.branch == 0 and det.gcafail == 0
    uo, un, mu = det.upar_old, det.upar_new, det.mu
    a = np.dot(fr0["vE"], fr0["bgb"])
    g = np.dot(fr0["vE"], fr0["vgb"])
    # Eq. (dupardtcase2disc)
    lhs = (un - uo) / dt
    rhs = (qm * np.dot(fr0["E"], fr0["b"]) + 0.5 * (uo + un) * a
           + 0.5 * (Gam(fr0, uo, mu) + Gam(fr0, un, mu)) * g)
    assert lhs == pytest.approx(rhs, abs=1e-7 * (1 + abs(rhs)))
    # the quadratic root is Gamma(R^n, u_par^{n+1/2}) of Eq. (lfacgca2)
    assert det.Gamma1 == pytest.approx(Gam(fr0, un, mu), rel=1e-12)
    # Eq. (dRdtcase2disc) at the returned R^{n+1}
    R1 = Rn + dxp
    fr1 = frame_fd(f, p, R1)
    H = R1 - Rn - 0.5 * dt * (Vgc(fr0, qm, un, mu) + Vgc(fr1, qm, un, mu))
    assert np.max(np.abs(H)) < 1e-8
    # decomposition at R^{n-1/2} (= R^n here) of Sec. 3.1
    G_full = gamma_of(u)
    assert uo == pytest.approx(np.dot(u, fr0["b"]), abs=1e-13)
    ug = u - uo * fr0["b"] - (fr0["vE"] + vcurv(fr0, qm, uo, G_full)) * G_full
    assert mu == pytest.approx(np.dot(ug, ug) / (2 * fr0["Bm"] * fr0["kappa"]), rel=1e-7)
    # reconstruction at R^{n+1/2} (Sec. 3.1)
    frh = frame_fd(f, p, Rn + 0.5 * dxp)
    Gh = Gam(frh, un, mu)
    uperp = math.sqrt(2 * mu * frh["Bm"] * frh["kappa"])
    want = un * frh["b"] + (frh["vE"] + vcurv(frh, qm, un, Gh)) * Gh + uperp * unit(ug)
    assert np.allclose(u2, want, atol=1e-7, rtol=0)


def test_gca_fixed_point_converges_in_few_iterations():
    """3-4 iterations reach an absolute iteration error of 1e-7 (Sec. 2.2.2)
    for a drift step through a field that varies over ~100 cells, as a PiC
    field does (the count includes the explicit first iterate)."""
    f = O.rotor_field(1.0, 0.05, 0.4)
    p = O.make_params(dt=0.45, qm=(-50.0,), force=O.FORCE_GCA, curvature=1, tol=1e-7,
                      max_iter=16)
    rng = np.random.default_rng(3)
    its = []
    for _ in range(20):
        R = rng.uniform(0, 10, size=3)
        u = rng.normal(size=3) * 0.5
        _, _, _, fl, det = O.step_one(f, p, R, u, np.zeros(3), 0)
        assert det.branch == 0 and not det.nonconv
        assert det.resid < 1e-7
        its.append(det.iters)
    assert max(its) <= 4


def test_harris_drift_closed_form():
    """Harris sheet B = (B0 tanh(y/delta), 0, Bg), E = Ez z: v_E = Ez Bx/B^2 y-hat,
    (b.grad)b = 0 and, writing b = (cos phi, 0, sin phi), the curvature drift is
    v_c = -(c kappa^2 / (q B)) u_par v_E,y phi'(y) y-hat with phi' = -Bg Bx'/B^2."""
    B0, delta, Bg, Ez, qm = 1.0, 4.0, 0.1, 0.05, -100.0
    f = O.harris_field(B0, delta, Bg, Ez)

    def closed(R, upar, mu):
        y = R[1]
        Bx = B0 * math.tanh(y / delta)
        dBx = B0 / delta / math.cosh(y / delta) ** 2
        B2 = Bx * Bx + Bg * Bg
        Bm = math.sqrt(B2)
        vEy = Ez * Bx / B2
        kappa = 1 / math.sqrt(1 - vEy ** 2)
        G = kappa * math.sqrt(1 + upar ** 2 + 2 * mu * Bm * kappa)
        phip = -Bg * dBx / B2
        vcy = -(kappa ** 2 / (qm * Bm)) * upar * vEy * phip
        return np.array([upar * Bx / Bm / G, vEy + vcy]), vcy

    R0 = np.array([3.0, 2.0])
    for dt in (0.02, 0.01):
        res = {}
        for curv in (0, 1):
            p = O.make_params(dt=dt, qm=(qm,), force=O.FORCE_GCA, curvature=curv,
                              fixed_iters=20)
            u = np.array([0.6, 0.02, 0.5])
            x2, u2, dxp, fl, det = O.step_one(f, p, R0, u, np.zeros(2), 0)
            # E_par kick: u_par += q dt Ez b_z / m with (b.grad)b = v_E.(v_E.grad)b = 0
            Bx = B0 * math.tanh(R0[1] / delta)
            bz = Bg / math.hypot(Bx, Bg)
            assert det.upar_new == pytest.approx(det.upar_old + qm * dt * Ez * bz, abs=1e-12)
            V, vcy = closed(R0 + 0.5 * dxp, det.upar_new, det.mu)
            if curv == 0:
                V = V - np.array([0.0, vcy])
            res[curv] = (dxp / dt, V, vcy)
        (V0, W0, _), (V1, W1, vcy) = res[0], res[1]
        assert abs(vcy) > 1e-5
        assert np.max(np.abs(V1 - W1)) < 50 * dt * dt * 1e-3 + 1e-12
        assert np.max(np.abs(V0 - W0)) < 50 * dt * dt * 1e-3 + 1e-12
        assert (V1 - V0)[1] == pytest.approx(vcy, rel=1e-3)


# --------------------------------------------------------------------------
# Conversions (Sec. 3.1)
# --------------------------------------------------------------------------
def test_decompose_reconstruct_round_trip_exact():
    """Without curvature drift, and with u_perp,g perpendicular to v_E, the
    assumption Gamma(R, u_par) = Gamma(full u) is exact (Gamma^2 (1 - v_E^2) =
    1 + u_par^2 + u_perp,g^2), so reconstruct(decompose(u)) = u at one point."""
    rng = np.random.default_rng(11)
    ny, nx = 32, 16
    y = (np.arange(ny) - ny / 2)[:, None] * np.ones((1, nx))
    E = [np.zeros((ny, nx)), np.zeros((ny, nx)), np.full((ny, nx), 0.05)]
    B = [np.tanh(y / 4.0), 0.02 * np.ones((ny, nx)), np.full((ny, nx), 0.1)]
    f = O.grid_field(E, B, (1.0, 1.0))
    p = O.make_params(dt=0.45, curvature=0)
    for _ in range(10):
        R = rng.uniform(0, 16, size=2)
        F = O.eval_field(f, p, R)
        b = unit(F[3:6])
        vE = np.cross(F[0:3], F[3:6]) / np.dot(F[3:6], F[3:6])
        kap = 1 / math.sqrt(1 - np.dot(vE, vE))
        upar, uperp = rng.normal(), abs(rng.normal())
        ch = unit(np.cross(b, vE))
        G = kap * math.sqrt(1 + upar ** 2 + uperp ** 2)
        u = upar * b + vE * G + uperp * ch
        ok, up, mu, upp, bpg = O.decompose(f, p, -1.0, R, u)
        assert ok and up == pytest.approx(upar, abs=1e-13)
        assert upp == pytest.approx(uperp, abs=1e-12)
        ok, u2 = O.reconstruct(f, p, -1.0, R, up, mu, upp, bpg)
        assert ok and np.allclose(u2, u, atol=1e-13 * (1 + np.linalg.norm(u)), rtol=0)


def test_gca_step_uses_staggered_midpoints():
    """The decomposition is taken at R^{n-1/2} = (R^n + R^{n-1})/2 = x - dxp/2
    and the reconstruction at R^{n+1/2} = (R^{n+1} + R^n)/2 (Sec. 3.1)."""
    f = O.rotor_field(1.0, 0.3, 0.4)
    p = O.make_params(dt=0.9, qm=(-8.0,), force=O.FORCE_GCA, curvature=1, fixed_iters=30)
    x = np.array([1.1, 0.4, -0.3])
    dxp = np.array([0.35, -0.2, 0.1])
    u = np.array([0.4, -0.6, 0.3])
    x2, u2, dxp2, fl, det = O.step_one(f, p, x, u, dxp, 0)
    ok, up, mu, upp, bpg = O.decompose(f, p, -8.0, x - 0.5 * dxp, u)
    assert det.upar_old == pytest.approx(up, abs=1e-14)
    assert det.mu == pytest.approx(mu, rel=1e-13)
    ok, want = O.reconstruct(f, p, -8.0, x + 0.5 * dxp2, det.upar_new, det.mu, det.uperp, bpg)
    assert np.allclose(u2, want, atol=1e-14, rtol=0)
    assert np.allclose(x2, x + dxp2, atol=1e-15, rtol=0)


def test_gca_E0_keeps_upar_and_passes_through_bottle():
    """E = 0: v_E = 0, so the GCA step keeps u_par exactly (mirror force is
    dropped in the reduced system, Sec. 2.2): the guiding center crosses the
    bottle that reflects the Boris particle."""
    B0, L = 1.0, 4.0
    f = O.bottle_field(B0, L)
    qm = 50.0
    p = O.make_params(dt=0.2, qm=(qm,), force=O.FORCE_GCA, curvature=1, fixed_iters=8)
    pitch = math.radians(50.0)
    u = np.array([0.5 * math.sin(pitch), 0.0, 0.5 * math.cos(pitch)])
    x, dxp = np.array([0.0, 0.0, -6.0]), np.zeros(3)
    for _ in range(400):
        x, u, dxp, _, det = O.step_one(f, p, x, u, dxp, 0)
        assert det.upar_new == det.upar_old
        if x[2] > 6.0:
            break
    assert x[2] > 6.0


def test_uperp_mode_conserves_energy_on_straight_lines():
    """mu_mode = UPERP_CONSERVE holds u_perp,g fixed, so with E = 0 and straight
    field lines Gamma is conserved exactly; mu_mode = MU_CONSERVE instead keeps
    u_perp,g^2 / B (Sec. 2.2)."""
    ny, nx = 8, 16
    X = np.arange(nx)[None, :] * np.ones((ny, 1))
    Bz = 1.0 + 0.5 * np.sin(2 * np.pi * X / nx)
    Z = np.zeros((ny, nx))
    f = O.grid_field([Z, Z, Z], [Z, Z, Bz], (1.0, 1.0))
    u = np.array([0.3, 0.4, 0.2])
    for mode in (O.UPERP_CONSERVE, O.MU_CONSERVE):
        p = O.make_params(dt=0.45, qm=(-40.0,), force=O.FORCE_GCA, mu_mode=mode)
        x2, u2, dxp2, fl, det = O.step_one(f, p, np.array([3.3, 1.0]), u, np.array([0.3, 0.0]), 0)
        F0 = O.eval_field(f, p, [3.3 - 0.15, 1.0])
        F1 = O.eval_field(f, p, [3.3 + 0.5 * dxp2[0], 1.0 + 0.5 * dxp2[1]])
        assert np.allclose(dxp2, 0.0, atol=1e-15)   # no drift: b = z, E = 0
        up0 = np.hypot(u[0], u[1])
        up1 = np.hypot(u2[0], u2[1])
        if mode == O.UPERP_CONSERVE:
            assert np.linalg.norm(u2) == pytest.approx(np.linalg.norm(u), rel=1e-14)
        else:
            assert up1 ** 2 / F1[5] == pytest.approx(up0 ** 2 / F0[5], rel=1e-13)
    # here the two points coincide since the guiding center does not move


# --------------------------------------------------------------------------
# Units: every factor of c is pinned by an exact scaling symmetry.
# c -> 2c, u -> 2u, E -> 2E, B -> 2B, lengths -> 2 lengths, t and q/m fixed.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("force", [O.FORCE_NONE, O.FORCE_BORIS, O.FORCE_GCA])
def test_speed_of_light_scaling_symmetry(force):
    rng = np.random.default_rng(2)
    ny, nx = 12, 10
    E = [rng.normal(size=(ny, nx)) * 0.05 for _ in range(3)]
    B = [rng.normal(size=(ny, nx)) * 0.3 + (1.0 if k == 2 else 0.0) for k in range(3)]
    lam = 2.0
    res = []
    for s in (1.0, lam):
        f = O.grid_field([s * e for e in E], [s * b for b in B], (s * 0.8, s * 1.1))
        p = O.make_params(c=s, dt=0.3, dl=s * 0.8, qm=(-6.0,), force=force, curvature=1,
                          fixed_iters=5)
        st = dict(x=np.array([[3.1, 5.7, 0.2], [2.2, 9.9, 4.4]]) * s,
                  u=np.array([[0.3, -0.2, 0.05], [0.1, 0.4, -0.3], [0.2, 0.0, 0.6]]) * s,
                  dxp=np.array([[0.1, -0.05, 0.0], [0.02, 0.1, -0.1]]) * s,
                  flags=np.zeros(3, np.uint8))
        stats = O.push_sr(st, f, p, 4)
        res.append((st, stats))
    (a, sa), (b, sb) = res
    assert np.array_equal(a["flags"], b["flags"])
    assert sa["n_gca"] == sb["n_gca"] and sa["n_boris"] == sb["n_boris"]
    for k in ("x", "u", "dxp"):
        assert np.allclose(lam * a[k], b[k], rtol=1e-13, atol=1e-13)


# --------------------------------------------------------------------------
# The coupled method against the gyro-resolved Boris reference (Sec. 4.1)
# --------------------------------------------------------------------------
def test_gca_tracks_resolved_boris_in_harris_sheet():
    B0, delta, Bg, Ez, qm = 1.0, 4.0, 0.1, 0.05, -2000.0
    f = O.harris_field(B0, delta, Bg, Ez)
    y0 = 6.0
    Bx = B0 * math.tanh(y0 / delta)
    B = np.array([Bx, 0.0, Bg])
    vE = np.cross([0, 0, Ez], B) / np.dot(B, B)
    u0 = vE / math.sqrt(1 - np.dot(vE, vE)) + 0.2 * unit(B)
    T = 20.0
    pg = O.make_params(dt=0.45, qm=(qm,), force=O.FORCE_GCA, curvature=1, tol=1e-10)
    x, u, dxp = np.array([0.0, y0]), u0.copy(), np.zeros(2)
    for _ in range(int(round(T / 0.45))):
        x, u, dxp, _, _ = O.step_one(f, pg, x, u, dxp, 0)
    t_gca = round(T / 0.45) * 0.45
    st = dict(x=np.array([[0.0], [y0]]), u=u0.reshape(3, 1).copy(), flags=np.zeros(1, np.uint8))
    pr = O.make_params(dt=0.45, qm=(qm,))
    O.push_resolved(st, f, pr, t_gca, 0.45)
    xr = st["x"][:, 0]
    disp = np.linalg.norm(x - np.array([0.0, y0]))
    assert disp > 1.0
    rho = np.linalg.norm(u0) / (abs(qm) * np.linalg.norm(B))
    assert np.linalg.norm(x - xr) < 5e-3 * disp + 5 * rho


# --------------------------------------------------------------------------
# Coupled step bookkeeping: flags, statistics, wrap, fallbacks
# --------------------------------------------------------------------------
def harris_grid(nx=32, ny=32, delta=4.0, Bg=0.1, Ez=0.05):
    y = (np.arange(ny) - ny // 2)[:, None] * np.ones((1, nx))
    Z = np.zeros((ny, nx))
    return O.grid_field([Z, Z, np.full((ny, nx), Ez)],
                        [np.tanh(y / delta), Z, np.full((ny, nx), Bg)], (1.0, 1.0))


def test_push_bookkeeping_and_wrap():
    f = harris_grid()
    rng = np.random.default_rng(4)
    n = 200
    st = dict(x=rng.uniform(0, 32, size=(2, n)), u=rng.normal(size=(3, n)) * 0.3,
              dxp=np.zeros((2, n)), flags=np.zeros(n, np.uint8))
    st["flags"][::2] |= 1 << 6         # species 1
    st["u"][0, 7] = np.nan             # frozen particle
    p = O.make_params(dt=0.45, qm=(-10.0, 10.0), curvature=1, tol=1e-9)
    ref = {k: v.copy() for k, v in st.items()}
    stats = O.push_sr(st, f, p, 3)
    assert stats["n_boris"] + stats["n_gca"] == 3 * (n - 1)
    assert stats["n_nonfinite"] == 3
    assert stats["n_gca"] > 0 and stats["n_boris"] > 0
    assert np.all((st["x"] >= 0) & (st["x"] < 32))
    assert (st["flags"][7] & O.FLAG_NONFINITE) and np.isnan(st["u"][0, 7])
    assert np.array_equal(st["flags"] >> 6, ref["flags"] >> 6)
    # replay particle by particle and check S bits, transitions and the wrap
    tg = tb = 0
    for i in range(n):
        if i == 7:
            continue
        x, u, d, fl = ref["x"][:, i], ref["u"][:, i], ref["dxp"][:, i], int(ref["flags"][i])
        for s in range(3):
            prev = fl & 1
            x2, u, d, fl, det = O.step_one(f, p, x, u, d, fl)
            assert (fl & 1) == det.S and ((fl >> 1) & 1) == prev
            tg += prev == 1 and det.S == 0
            tb += prev == 0 and det.S == 1
            unwrapped = x + d
            assert np.allclose(x2, np.mod(unwrapped, 32.0), atol=1e-12)
            x = x2
        assert np.allclose(x, st["x"][:, i], atol=0, rtol=0)
        assert np.array_equal(u, st["u"][:, i])
    assert tg == stats["n_to_gca"] and tb == stats["n_to_boris"]


def test_quadratic_failure_falls_back_to_boris():
    """A curvature acceleration so under-resolved that the quadratic has no
    root >= 1 (k1 >= 0) makes the step a Boris step, flagged GCAFAIL."""
    f = O.rotor_field(1.0, 0.3, 0.9)
    x = np.array([0.05, 0.0, 0.0])
    u = np.array([0.1, 0.2, 0.3])
    pg = O.make_params(dt=60.0, qm=(-1e4,), force=O.FORCE_GCA, curvature=1, fixed_iters=3)
    pb = O.make_params(dt=60.0, qm=(-1e4,), force=O.FORCE_BORIS, curvature=1)
    x1, u1, d1, fl1, det1 = O.step_one(f, pg, x, u, np.zeros(3), 0)
    x2, u2, d2, fl2, det2 = O.step_one(f, pb, x, u, np.zeros(3), 0)
    assert det1.k1 >= 0 and det1.gcafail == 1 and (fl1 & O.FLAG_GCAFAIL)
    assert np.array_equal(u1, u2) and np.array_equal(x1, x2)


def test_nonconvergence_is_flagged():
    f = O.rotor_field(1.0, 0.3, 0.4)
    p = O.make_params(dt=0.45, qm=(-50.0,), force=O.FORCE_GCA, curvature=1, tol=1e-30,
                      max_iter=2)
    _, _, _, fl, det = O.step_one(f, p, np.array([1.0, 2.0, 3.0]), np.array([0.3, 0.2, 0.1]),
                                  np.zeros(3), 0)
    assert det.nonconv == 1 and det.iters == 2 and (fl & O.FLAG_NONCONV)
