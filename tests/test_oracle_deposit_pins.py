"""Pins of the oracle's current deposition (PiC coupling, Sec. 1 and 5: the
coupled scheme returns x and u at the usual staggered times, so a PiC code
deposits each step's current as for any particle).  The oracle's reading: a
cloud-in-cell cloud moving along the straight path x^n -> x^{n+1} at the
step's constant velocity, J the exact time average of its current on the
staggered points.

- Discrete continuity: with the cloud-in-cell charge rho (computed here from
  the hat weights), (rho^{n+1} - rho^n)/dt + div J = 0 to rounding, for paths
  crossing several cells along every axis, across the periodic edges, in 2D
  and 3D with unequal cell sizes.
- Brute force: the defining time integral sampled at 2e5 points of one step
  (box and hat functions evaluated directly) for every staggered point.
- Moments: sum J V = Q w v (every component), and the first moment of J along
  an axis other than its own equals Q w v times the path's midpoint (hats
  reproduce linear functions; the time average of a linear path is its
  midpoint).
- A particle at rest deposits no in-plane current; its 2D out-of-plane
  current is Q w v_z times its cloud-in-cell weights.
- The push: the current of a step equals Q w times the step's velocity, in
  uniform fields the closed form of each branch (Boris: u^{n+1/2}/Gamma;
  guiding center: u_par b/Gamma + v_E); species charges and weights; paths
  longer than the cap are left out and counted.
"""
import math

import numpy as np
import pytest

import oracle as O


def hat(s):
    return np.maximum(0.0, 1.0 - np.abs(s))


def cic_rho(x, q, n, dx):
    """rho at the nodes of a periodic grid from the hat weights (x: (nd, m))."""
    nd = len(n)
    rho = np.zeros(tuple(reversed(n)))
    V = float(np.prod(dx))
    for p in range(x.shape[1]):
        s = [x[a, p] / dx[a] for a in range(nd)]
        base = [math.floor(v) for v in s]
        for o in range(1 << nd):
            idx, w = [], q[p] / V
            for a in range(nd):
                node = base[a] + ((o >> a) & 1)
                w *= hat(s[a] - node)
                idx.append(node % n[a])
            rho[tuple(reversed(idx))] += w
    return rho


def div_J(J, n, dx):
    """Backward-difference divergence of the staggered J at the nodes."""
    nd = len(n)
    out = np.zeros_like(J[0])
    for a in range(nd):
        ax = nd - 1 - a                     # numpy axis of grid axis a
        out += (J[a] - np.roll(J[a], 1, axis=ax)) / dx[a]
    return out


def grid(n, dx):
    shape = tuple(reversed(n))
    z = np.zeros(int(np.prod(n)))
    return O.OracleField(O.FIELD_GRID, len(n), n, dx, E=[z] * 3, B=[z + 1.0] * 3), shape


@pytest.mark.parametrize("nd", [2, 3])
def test_discrete_continuity(nd):
    rng = np.random.default_rng(40 + nd)
    n = (7, 5, 4)[:nd]
    dx = (0.8, 1.3, 0.6)[:nd]
    f, shape = grid(n, dx)
    m, dt = 60, 0.37
    L = np.array(n) * np.array(dx)
    x0 = rng.uniform(0, 1, (nd, m)) * L[:, None]
    x0[:, :10] = (L[:, None] - 0.05 * np.array(dx)[:, None])     # next to the far edge
    disp = rng.uniform(-3.2, 3.2, (nd, m)) * np.array(dx)[:, None]
    disp[0, 10:14] = 0.0                                         # along a face of axis 0
    x0[1, 12:14] = 2.0 * dx[1]
    q = rng.uniform(-2, 2, m)
    cur = O.Current(shape, q=(1.0,))
    for p in range(m):
        assert O.deposit(f, x0[:, p], disp[:, p], 0.3, q[p], dt, cur)
    x1 = np.mod(x0 + disp, L[:, None])
    r0, r1 = cic_rho(x0, q, n, dx), cic_rho(x1, q, n, dx)
    res = (r1 - r0) / dt + div_J(cur.J, n, dx)
    scale = np.abs(r0).max() / dt + max(np.abs(cur.J[a]).max() / dx[a] for a in range(nd))
    assert np.abs(res).max() < 1e-13 * scale, np.abs(res).max() / scale


def brute_force(x0, disp, vz, Qw, dt, n, dx, N=200000):
    """The definition sampled at N midpoints of the step."""
    nd = len(n)
    V = float(np.prod(dx))
    t = (np.arange(N) + 0.5) / N
    s = [(x0[a] + disp[a] * t) / dx[a] for a in range(nd)]
    J = [np.zeros(tuple(reversed(n))) for _ in range(3)]
    for comp in range(3):
        vel = disp[comp] / dt if comp < nd else vz
        for node in np.ndindex(*reversed(n)):
            idx = list(reversed(node))
            g = np.ones(N)
            for b in range(nd):
                # images of the node under the periodic wrap that the path can reach
                k = np.round((s[b] - idx[b]) / n[b]) * n[b] + idx[b]
                if b == comp:
                    g *= ((s[b] - k) >= 0) & ((s[b] - k) < 1)     # Pi(s - i - 1/2)
                else:
                    g *= hat(s[b] - k)
            J[comp][node] = Qw * vel * g.mean() / V
    return J


@pytest.mark.parametrize("nd,x0,disp", [
    (2, (1.3, 2.2), (2.45, -1.7)),
    (2, (6.9, 0.1), (0.8, -0.35)),          # across both periodic edges
    (3, (1.2, 0.7, 2.1), (1.6, 0.9, -1.3)),
    (3, (0.4, 3.9, 0.2), (-0.9, 0.45, 0.0)),
])
def test_brute_force_time_integral(nd, x0, disp):
    n = (8, 5, 4)[:nd]
    dx = (1.0, 1.0, 1.0)[:nd] if nd == 3 else (1.0, 1.1)
    f, shape = grid(n, dx)
    dt, vz, Qw = 0.45, -0.3, 1.7
    cur = O.Current(shape, q=(1.0,))
    assert O.deposit(f, np.array(x0), np.array(disp), vz, Qw, dt, cur)
    want = brute_force(np.array(x0), np.array(disp), vz, Qw, dt, n, dx)
    for a in range(3):
        tot = np.abs(want[a]).sum() + 1e-30
        assert np.abs(cur.J[a] - want[a]).max() < 2e-5 * tot, (a, np.abs(cur.J[a] - want[a]).max())


@pytest.mark.parametrize("nd", [2, 3])
def test_moments(nd):
    rng = np.random.default_rng(7 + nd)
    n = (16, 14, 12)[:nd]
    dx = (0.7, 1.2, 0.9)[:nd]
    f, shape = grid(n, dx)
    V = float(np.prod(dx))
    dt = 0.4
    for _ in range(10):
        # interior paths, so that node coordinates need no unwrapping
        x0 = np.array([rng.uniform(4, 7) * dx[a] for a in range(nd)])
        disp = rng.uniform(-2.5, 2.5, nd) * np.array(dx)
        vz, Qw = rng.normal(), rng.uniform(0.5, 2)
        cur = O.Current(shape, q=(1.0,))
        assert O.deposit(f, x0, disp, vz, Qw, dt, cur)
        xm = x0 + 0.5 * disp
        for a in range(3):
            v = disp[a] / dt if a < nd else vz
            assert cur.J[a].sum() * V == pytest.approx(Qw * v, rel=1e-12, abs=1e-14)
            for b in range(nd):
                if b == a:
                    continue
                coord = np.arange(n[b]) * dx[b]
                shp = [1] * nd
                shp[nd - 1 - b] = n[b]
                mom = (cur.J[a] * coord.reshape(shp)).sum() * V
                assert mom == pytest.approx(Qw * v * xm[b], rel=1e-11, abs=1e-13)


def test_particle_at_rest():
    n, dx = (6, 5), (1.0, 2.0)
    f, shape = grid(n, dx)
    x0 = np.array([2.25, 4.5])
    cur = O.Current(shape, q=(1.0,))
    assert O.deposit(f, x0, np.zeros(2), 0.6, 2.0, 0.5, cur)
    assert not cur.J[0].any() and not cur.J[1].any()
    want = np.zeros(shape)
    want[2, 2], want[2, 3], want[3, 2], want[3, 3] = 0.75 * 0.75, 0.25 * 0.75, 0.75 * 0.25, 0.25 * 0.25
    assert np.allclose(cur.J[2], 2.0 * 0.6 * want / 2.0, rtol=0, atol=1e-15)


def uniform_grid_field(E, B, n=(12, 10)):
    shape = tuple(reversed(n))
    ones = np.ones(int(np.prod(n)))
    return O.OracleField(O.FIELD_GRID, 2, n, (1.0, 1.0), E=[e * ones for e in E],
                         B=[b * ones for b in B]), shape


def test_push_current_matches_branch_closed_forms():
    """Uniform E normal to B, B with an out-of-plane part: guiding-center
    particles (forced) deposit Q w (u_par b/Gamma + v_E), Boris particles
    Q w u^{n+1/2}/Gamma; two species with their charges and weights."""
    E, B = np.array([0.0, 0.1, 0.0]), np.array([0.3, 0.0, 1.0])
    f, shape = uniform_grid_field(E, B)
    rng = np.random.default_rng(5)
    m, dt = 40, 0.45
    Bm = np.linalg.norm(B)
    b = B / Bm
    vE = np.cross(E, B) / (B @ B)
    kappa = 1.0 / math.sqrt(1.0 - vE @ vE)
    for force in (O.FORCE_GCA, O.FORCE_BORIS):
        x = rng.uniform(1, 9, (2, m))
        u = rng.normal(0, 0.5, (3, m))
        st = dict(x=x.copy(), u=u.copy(), dxp=np.zeros((2, m)),
                  flags=((np.arange(m) % 2) << 6).astype(np.uint8))
        w = rng.uniform(0.5, 1.5, m)
        p = O.make_params(dt=dt, qm=(-30.0, 30.0), force=force, fixed_iters=4, curvature=1)
        cur = O.Current(shape, q=(-1.0, 2.0), w=w)
        O.push_sr(st, f, p, 1, current=cur)
        Qw = np.where(np.arange(m) % 2 == 0, -1.0, 2.0) * w
        if force == O.FORCE_BORIS:
            G = np.sqrt(1.0 + (st["u"] ** 2).sum(0))
            v = st["u"] / G
        else:
            qm = np.where(np.arange(m) % 2 == 0, -30.0, 30.0)
            G0 = np.sqrt(1.0 + (u ** 2).sum(0))
            upar0 = b @ u
            ug = u - np.outer(b, upar0) - np.outer(vE, G0)
            mu = (ug ** 2).sum(0) / (2.0 * Bm * kappa)
            upar1 = upar0 + qm * dt * (E @ b)
            G1 = kappa * np.sqrt(1.0 + upar1 ** 2 + 2.0 * mu * Bm * kappa)
            v = np.outer(b, upar1 / G1) + vE[:, None]
            assert np.allclose(st["dxp"], dt * v[:2], rtol=0, atol=1e-13)
        for a in range(3):
            assert cur.J[a].sum() == pytest.approx((Qw * v[a]).sum(), rel=1e-12, abs=1e-14)
        assert cur.n_skipped == 0
        # the current is that of the step's own path: continuity with the
        # charge before and after the push
        n, dx = (12, 10), (1.0, 1.0)
        r0, r1 = cic_rho(x, Qw, n, dx), cic_rho(st["x"], Qw, n, dx)
        res = (r1 - r0) / dt + div_J(cur.J, n, dx)
        assert np.abs(res).max() < 1e-12 * (np.abs(r0).max() / dt)


def test_step_velocity_is_the_path_velocity():
    """In a non-uniform field (Harris sheet on a grid, coupled switch) every
    advanced particle's step velocity, whose out-of-plane component the 2D
    deposition uses, moves it by exactly its displacement: x^{n+1} - x^n =
    dt v_step in the plane, for both branches; frozen particles deposit
    nothing and the pushed current satisfies continuity."""
    from paper_2007_14401_gb300 import inputs
    fields, st, prm = inputs.harris_2d(nx=32, ny=32, n_per_species=100, seed=3)
    f = O.grid_field(fields["E"], fields["B"], fields["dx"])
    p = O.make_params(dt=prm["dt"], qm=prm["qm"], f_rho=prm["f_rho"], dl=prm["dl"],
                      fixed_iters=5)
    branches = set()
    for i in range(st["x"].shape[1]):
        x, u, d, fl, det = O.step_one(f, p, st["x"][:, i], st["u"][:, i], st["dxp"][:, i],
                                      int(st["flags"][i]))
        branches.add(det.branch)
        assert np.allclose(np.array(det.vstep[:2]) * prm["dt"], d, rtol=1e-13, atol=1e-15)
        if det.branch == 1:
            G = math.sqrt(1.0 + u @ u)
            assert det.vstep[2] == pytest.approx(u[2] / G, rel=1e-14)
    assert branches == {0, 1}
    m = st["x"].shape[1]
    s2 = {k: v.copy() for k, v in st.items()}
    s2["u"][:, 5] = np.nan
    x0 = s2["x"].copy()
    n = tuple(reversed(fields["E"][0].shape))
    cur = O.Current(fields["E"][0].shape, q=(1.0, -1.0))
    O.push_sr(s2, f, p, 1, current=cur)
    qs = np.array([1.0, -1.0, 0.0, 0.0])[(s2["flags"] >> 6) & 3]
    qs[5] = 0.0                                    # frozen: no charge moved, none deposited
    r0, r1 = cic_rho(x0, qs, n, fields["dx"]), cic_rho(s2["x"], qs, n, fields["dx"])
    res = (r1 - r0) / prm["dt"] + div_J(cur.J, n, fields["dx"])
    assert np.abs(res).max() < 1e-12 * (np.abs(r0).max() / prm["dt"])
    assert s2["flags"][5] & O.FLAG_NONFINITE and m > 100


def test_long_paths_are_left_out():
    n = (8, 8)
    f, shape = grid(n, (1.0, 1.0))
    cur = O.Current(shape, q=(1.0,))
    assert not O.deposit(f, np.array([1.0, 1.0]), np.array([O.DEP_MAX_CELLS + 0.5, 0.0]),
                         0.0, 1.0, 1.0, cur)
    assert not any(c.any() for c in cur.J)
    assert O.deposit(f, np.array([1.0, 1.0]), np.array([O.DEP_MAX_CELLS - 0.5, 0.0]),
                     0.0, 1.0, 1.0, cur)
    assert cur.J[0].sum() == pytest.approx(O.DEP_MAX_CELLS - 0.5, rel=1e-12)
