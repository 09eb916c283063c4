"""Seeded synthetic workloads shaped like the paper's current-sheet tests.

This module only builds inputs: fields on a periodic node grid and particle
states.  It holds none of the pusher's arithmetic, and it is the one module
both the CUDA path and the CPU oracle consume (the oracle through the test
suite).  Everything is generated in float64 with numpy's PCG64 generator from
an explicit seed; float32 copies are rounded from these arrays.

Layout of what is returned (the "plain" layout):
  fields:  dict(E=[Ex, Ey, Ez], B=[Bx, By, Bz], dB=None | [d_i B_j for i < ndim,
           j < 3] (i major), dx=(dx, dy[, dz])), each node array of shape
           (ny, nx) or (nz, ny, nx), node (i, j, k) at (i dx, j dy, k dz).
  state:   dict(x=(ndim, n), u=(3, n), dxp=(ndim, n) float64, flags=(n,) uint8)
           with x^0 in [0, L), u taken as u^{-1/2} and dxp = x^0 - x^{-1}.
  params:  dict of the pusher parameters of the workload.

The paper's own field snapshots (a TRISTAN-MP reconnection run and a GRPiC
black-hole run) are not available; these analytic fields stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

SPECIES_SHIFT = 6


# --------------------------------------------------------------------------
# momentum distributions
# --------------------------------------------------------------------------
def _isotropic(rng, n):
    mu = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(1.0 - mu * mu)
    return np.stack([s * np.cos(ph), s * np.sin(ph), mu])


def maxwell_juttner(rng, n, theta, c=1.0):
    """Momenta u = gamma v (units of c) from the Maxwell-Juttner distribution
    f(u) ~ u^2 exp(-gamma/theta), isotropic.  The kinetic energy e = gamma - 1
    has density ~ sqrt(e (e + 2)) (1 + e) exp(-e/theta); it is sampled by
    inverse transform on a tabulated CDF (2^20 trapezoid panels)."""
    emax = theta * 60.0 + 1.0
    e = np.linspace(0.0, emax, (1 << 20) + 1)
    pdf = np.sqrt(e * (e + 2.0)) * (1.0 + e) * np.exp(-e / theta)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(e))])
    cdf /= cdf[-1]
    ek = np.interp(rng.uniform(0.0, 1.0, n), cdf, e)
    umag = np.sqrt(ek * (ek + 2.0)) * c
    return _isotropic(rng, n) * umag


def power_law_gamma(rng, n, gmin, gmax, c=1.0):
    """Momenta with dN/dgamma ~ gamma^-2 on [gmin, gmax], isotropic
    (inverse CDF of the power law)."""
    U = rng.uniform(0.0, 1.0, n)
    g = 1.0 / (1.0 / gmin - U * (1.0 / gmin - 1.0 / gmax))
    umag = np.sqrt(np.maximum(g * g - 1.0, 0.0)) * c
    return _isotropic(rng, n) * umag


def initial_state(x, u, dt, species, c=1.0):
    """Pack a state: u is taken as u^{-1/2} and the previous displacement as
    dxp = dt u / gamma (the step that would have brought the particle to x)."""
    nd = x.shape[0]
    g = np.sqrt(1.0 + np.sum(u * u, axis=0) / (c * c))
    dxp = dt * u[:nd] / g
    flags = (np.asarray(species, dtype=np.uint8) << SPECIES_SHIFT).astype(np.uint8)
    return dict(x=np.ascontiguousarray(x, dtype=np.float64),
                u=np.ascontiguousarray(u, dtype=np.float64),
                dxp=np.ascontiguousarray(dxp, dtype=np.float64),
                flags=np.ascontiguousarray(flags))


def central_gradients(B, dx):
    """d_i B_j at the nodes by second-order periodic central differences
    (the precomputed gradient grids of the 2D reconnection workload)."""
    nd = B[0].ndim
    out = []
    for i in range(nd):
        axis = nd - 1 - i            # arrays are (.., y, x): x is the last axis
        for j in range(3):
            out.append((np.roll(B[j], -1, axis) - np.roll(B[j], 1, axis)) / (2.0 * dx[i]))
    return out


# --------------------------------------------------------------------------
# 2D Harris sheet, FP64 (4096 particles per charge-to-mass ratio)
# --------------------------------------------------------------------------
def harris_2d(nx=128, ny=128, dx=1.0, B0=1.0, delta=4.0, Bg=0.1, Ez=0.05,
              n_per_species=4096, qms=(-1.0, -10.0, -100.0, -1000.0), theta=0.1,
              dt=1.0, seed=0):
    """Single Harris sheet B_x = B0 tanh(y/delta), guide field Bg, uniform Ez,
    on y in [-ny/2, ny/2) (the periodic seam at y = +-ny/2 is a one-cell
    reversal), particles uniform in the box with Maxwell-Juttner momenta, one
    species per charge-to-mass ratio (the paper's sweep of q/m, Sec. 4.1)."""
    rng = np.random.default_rng(seed)
    y = (np.arange(ny) * dx - 0.5 * ny * dx)[:, None] * np.ones((1, nx))
    Z = np.zeros((ny, nx))
    fields = dict(E=[Z.copy(), Z.copy(), np.full((ny, nx), Ez)],
                  B=[B0 * np.tanh(y / delta), Z.copy(), np.full((ny, nx), Bg)],
                  dB=None, dx=(dx, dx))
    ns = len(qms)
    n = n_per_species * ns
    x = np.stack([rng.uniform(0.0, nx * dx, n), rng.uniform(0.0, ny * dx, n)])
    u = maxwell_juttner(rng, n, theta)
    species = np.repeat(np.arange(ns), n_per_species)
    state = initial_state(x, u, dt, species)
    params = dict(c=1.0, dt=dt, f_rho=0.4, f_E=1.0, dl=dx, qm=tuple(qms),
                  curvature=1, mu_mode=0, grad_mode=0, gca_max_iter=16,
                  gca_fixed_iters=0, gca_tol=1e-7, n_steps=1000)
    return fields, state, params


# --------------------------------------------------------------------------
# 2D reconnection-like field, mixed precision (FP32 fields + gradient grids)
# --------------------------------------------------------------------------
def reconnection_2d(nx=2048, ny=1024, dx=1.0, B0=1.0, delta=8.0, psi0=0.1,
                    n_modes=64, mode_amp=0.02, max_mode=16, vin=0.1,
                    n_particles=1 << 24, theta=1.0, dt=0.45, omega_dt_max=1e5,
                    seed=1, mode_amps=None):
    """Double Harris sheet B_x = B0[tanh((y+Ly/4)/d) - tanh((y-Ly/4)/d) - 1] on
    y in [-Ly/2, Ly/2), a GEM-style flux perturbation psi = psi0 cos(2 pi x/Lx)
    cos(pi y/Ly), n_modes random-phase Fourier modes of psi with |dB_m| =
    mode_amp, B += z x grad(psi), and E = -v_in x B with v_in = vin sin(4 pi
    y/Ly) y-hat (inflow toward both sheets).  Half positrons, half electrons,
    Maxwell-Juttner theta; |q/m| set so that max Omega_C dt = omega_dt_max.
    ``mode_amps`` overrides the 64 mode amplitudes (the adjoint workload)."""
    rng = np.random.default_rng(seed)
    Lx, Ly = nx * dx, ny * dx
    X = (np.arange(nx) * dx)[None, :] * np.ones((ny, 1))
    Y = (np.arange(ny) * dx - 0.5 * Ly)[:, None] * np.ones((1, nx))
    Bx = B0 * (np.tanh((Y + Ly / 4) / delta) - np.tanh((Y - Ly / 4) / delta) - 1.0)
    By = np.zeros_like(Bx)
    # z x grad(psi) = (-d_y psi, d_x psi, 0)
    kx0, ky0 = 2 * math.pi / Lx, math.pi / Ly
    Bx += psi0 * ky0 * np.cos(kx0 * X) * np.sin(ky0 * Y)
    By += -psi0 * kx0 * np.sin(kx0 * X) * np.cos(ky0 * Y)
    # mode numbers uniform on {-max_mode..max_mode} without 0
    nxm = rng.integers(1, max_mode, size=n_modes, endpoint=True) * rng.choice([-1, 1], n_modes)
    nym = rng.integers(1, max_mode, size=n_modes, endpoint=True) * rng.choice([-1, 1], n_modes)
    phase = rng.uniform(0.0, 2 * math.pi, n_modes)
    amps = np.full(n_modes, mode_amp) if mode_amps is None else np.asarray(mode_amps, float)
    for m in range(n_modes):
        kx, ky = 2 * math.pi * nxm[m] / Lx, 2 * math.pi * nym[m] / Ly
        k = math.hypot(kx, ky)
        s = np.sin(kx * X + ky * Y + phase[m])
        # psi_m = (a/k) cos(k.x + phi):  -d_y psi = (a/k) ky sin, d_x psi = -(a/k) kx sin
        Bx += amps[m] / k * ky * s
        By += -amps[m] / k * kx * s
    Bz = np.zeros_like(Bx)
    v = vin * np.sin(4 * math.pi * Y / Ly)
    # E = -v x B with v = v y-hat:  -(v Bz, 0, -v Bx)
    E = [-v * Bz, np.zeros_like(Bx), v * Bx]
    B = [Bx, By, Bz]
    fields = dict(E=E, B=B, dB=central_gradients(B, (dx, dx)), dx=(dx, dx),
                  modes=dict(nx=nxm, ny=nym, phase=phase, amp=amps))
    Bmax = float(np.sqrt(Bx * Bx + By * By + Bz * Bz).max())
    Q = omega_dt_max / (dt * Bmax)
    prng = np.random.default_rng(seed + 1000)
    x = np.stack([prng.uniform(0.0, Lx, n_particles), prng.uniform(0.0, Ly, n_particles)])
    u = maxwell_juttner(prng, n_particles, theta)
    species = (np.arange(n_particles) % 2).astype(np.uint8)   # 0 electron, 1 positron
    state = initial_state(x, u, dt, species)
    params = dict(c=1.0, dt=dt, f_rho=0.4, f_E=1.0, dl=dx, qm=(-Q, Q),
                  curvature=1, mu_mode=0, grad_mode=1, gca_max_iter=16,
                  gca_fixed_iters=0, gca_tol=1e-7, n_steps=500)
    return fields, state, params


def reconnection_2d_modes(**kw):
    """The reconnection workload split for differentiation with respect to the
    Fourier-mode amplitudes a_m: its fields are base + sum_m a_m pattern_m
    (B, E = -v_in x B and the central-difference gradients are all linear in
    the a_m).  Returns (base, patterns, amps, state, params): base and each
    pattern are field dicts (E, B, dB, dx) without particles; amps, state and
    params are those of reconnection_2d(**kw), so |q/m| stays fixed when the
    amplitudes move."""
    fields, state, params = reconnection_2d(**kw)
    md = fields["modes"]
    kz = dict(kw, n_particles=1, mode_amps=np.zeros(len(md["amp"])))
    base, _, _ = reconnection_2d(**kz)
    base.pop("modes")
    ny, nx = np.asarray(fields["B"][0]).shape
    dx = fields["dx"][0]
    Lx, Ly = nx * dx, ny * dx
    X = (np.arange(nx) * dx)[None, :] * np.ones((ny, 1))
    Y = (np.arange(ny) * dx - 0.5 * Ly)[:, None] * np.ones((1, nx))
    v = kw.get("vin", 0.1) * np.sin(4 * math.pi * Y / Ly)
    patterns = []
    for m in range(len(md["amp"])):
        kx, ky = 2 * math.pi * md["nx"][m] / Lx, 2 * math.pi * md["ny"][m] / Ly
        k = math.hypot(kx, ky)
        sn = np.sin(kx * X + ky * Y + md["phase"][m])
        Bx, By, Bz = ky / k * sn, -kx / k * sn, np.zeros_like(sn)
        B = [Bx, By, Bz]
        patterns.append(dict(E=[np.zeros_like(sn), np.zeros_like(sn), v * Bx], B=B,
                             dB=central_gradients(B, (dx, dx)), dx=(dx, dx)))
    return base, patterns, np.asarray(md["amp"], float), state, params


def combine_fields(base: dict, patterns: list, amps) -> dict:
    """base + sum_m amps[m] patterns[m], component by component."""
    def comb(key):
        out = []
        for c in range(len(base[key])):
            acc = np.array(base[key][c], dtype=np.float64, copy=True)
            for a, p in zip(amps, patterns):
                acc = acc + a * np.asarray(p[key][c])
            out.append(acc)
        return out
    return dict(E=comb("E"), B=comb("B"), dB=comb("dB"), dx=base["dx"])


# --------------------------------------------------------------------------
# 3D kinked current sheet, mixed precision
# --------------------------------------------------------------------------
def current_sheet_3d(n=256, dx=1.0, B0=1.0, delta=6.0, Bg=0.3, kink=0.05, Ey=0.1,
                     n_particles=1 << 26, frac_thermal=0.7, theta=0.3, gmax=1e4,
                     Q=20.0, dt=0.45, seed=2):
    """Harris sheet B_x = B0 tanh((y - y_c(z))/delta) with y_c(z) = kink Ly
    sin(2 pi z/Lz), guide field Bg along z and uniform E_y, y in [-L/2, L/2).
    70% of the particles are Maxwell-Juttner theta upstream (|y - y_c| >
    2 delta), 30% a gamma^-2 power law on [1, gmax] inside the sheet
    (|y - y_c| < delta); half positrons, half electrons, |q/m| = Q."""
    rng = np.random.default_rng(seed)
    L = n * dx
    z = (np.arange(n) * dx)[:, None, None]
    y = (np.arange(n) * dx - 0.5 * L)[None, :, None]
    yc = kink * L * np.sin(2 * math.pi * z / L)
    shape = (n, n, n)
    Bx = np.broadcast_to(B0 * np.tanh((y - yc) / delta), shape).astype(np.float64)
    Z = np.zeros(shape)
    fields = dict(E=[Z, np.full(shape, Ey), Z], B=[Bx, Z, np.full(shape, Bg)],
                  dB=None, dx=(dx, dx, dx))
    n_th = int(round(frac_thermal * n_particles))
    n_pl = n_particles - n_th
    prng = np.random.default_rng(seed + 1000)

    def place(count, inside):
        xs = np.empty((3, 0))
        while xs.shape[1] < count:
            m = 2 * (count - xs.shape[1]) + 1024
            c = np.stack([prng.uniform(0, L, m), prng.uniform(0, L, m), prng.uniform(0, L, m)])
            d = np.abs(c[1] - 0.5 * L - kink * L * np.sin(2 * math.pi * c[2] / L))
            keep = d < delta if inside else d > 2 * delta
            xs = np.concatenate([xs, c[:, keep]], axis=1)
        return xs[:, :count]

    x = np.concatenate([place(n_th, False), place(n_pl, True)], axis=1)
    u = np.concatenate([maxwell_juttner(prng, n_th, theta),
                        power_law_gamma(prng, n_pl, 1.0, gmax)], axis=1)
    species = (np.arange(n_particles) % 2).astype(np.uint8)
    state = initial_state(x, u, dt, species)
    params = dict(c=1.0, dt=dt, f_rho=0.4, f_E=1.0, dl=dx, qm=(-Q, Q),
                  curvature=1, mu_mode=0, grad_mode=0, gca_max_iter=16,
                  gca_fixed_iters=0, gca_tol=1e-7, n_steps=200)
    return fields, state, params


def subset(state, idx):
    """The particles ``idx`` of a state (copies)."""
    return {k: np.ascontiguousarray(v[..., idx]) for k, v in state.items()}


# --------------------------------------------------------------------------
# Kerr black hole: Wald field plus a split monopole (covariant scheme)
# --------------------------------------------------------------------------
def _ks_line_element(a, r, th):
    """Kerr metric in Kerr-Schild coordinates (t, r, theta, phi), M = 1:
    g_{mu nu} for arrays r, th (shape (..., 4, 4))."""
    s, c = np.sin(th), np.cos(th)
    rho2 = r * r + a * a * c * c
    z = 2.0 * r / rho2
    g = np.zeros(np.shape(r) + (4, 4))
    g[..., 0, 0] = -(1.0 - z)
    g[..., 0, 1] = g[..., 1, 0] = z
    g[..., 0, 3] = g[..., 3, 0] = -a * z * s * s
    g[..., 1, 1] = 1.0 + z
    g[..., 1, 3] = g[..., 3, 1] = -a * (1.0 + z) * s * s
    g[..., 2, 2] = rho2
    g[..., 3, 3] = (r * r + a * a + z * a * a * s * s) * s * s
    return g


def kerr_wald(nr=512, nth=512, a=0.9, B0=1.0, Qm=1.0, r_out=50.0, n_particles=1 << 22,
              theta_mj=1.0, qm=-1e3, dt=0.02, seed=4):
    """Kerr-Schild grid uniform in (log r, theta), r in [1.2 r_h, r_out], theta
    in [0, pi] (nodes on the poles).  Field: Wald's uniform-at-infinity
    solution A_mu = (B0/2)(g_{mu phi} + 2 a g_{mu t}) (Wald 1974) plus a split
    monopole A_phi = -Qm s(theta) cos(theta), s a sign of cos(theta) smoothed
    over two cells, whose reversal is an equatorial current sheet.  D^i =
    alpha F^{t i}, B^i = epsilon^{ijk} F_jk / (2 sqrt(gamma)), contravariant
    Kerr-Schild components, derivatives of A by central differences.
    Electrons uniform in (log r, theta, phi), Maxwell-Juttner momenta in the
    frame of the normal observer (triad from the Cholesky factor of gamma^{ij})."""
    rh = 1.0 + np.sqrt(1.0 - a * a)
    r_in = 1.2 * rh
    logr0 = np.log(r_in)
    dlogr = (np.log(r_out) - logr0) / (nr - 1)
    dth = np.pi / (nth - 1)
    R = np.exp(logr0 + dlogr * np.arange(nr))[None, :] * np.ones((nth, 1))
    # the metric is singular on the axis: evaluate the pole rows just off it
    # (they are replaced by the neighbouring rows below)
    T = np.clip((dth * np.arange(nth))[:, None] * np.ones((1, nr)), 0.25 * dth, np.pi - 0.25 * dth)
    w = 2.0 * dth

    def potential(r, th):
        g = _ks_line_element(a, r, th)
        A = 0.5 * B0 * (g[..., :, 3] + 2.0 * a * g[..., :, 0])
        A[..., 3] += -Qm * np.tanh(np.cos(th) / w) * np.cos(th)
        return A

    hr, ht = 1e-6 * R, 1e-6
    dA_r = (potential(R + hr, T) - potential(R - hr, T)) / (2 * hr)[..., None]
    Tp, Tm = T + ht, T - ht
    dA_t = (potential(R, Tp) - potential(R, Tm)) / (Tp - Tm)[..., None]
    F = np.zeros((nth, nr, 4, 4))
    for mu, dA in ((1, dA_r), (2, dA_t)):      # F_{mu nu} = d_mu A_nu - d_nu A_mu
        F[..., mu, :] += dA
        F[..., :, mu] -= dA
    g4 = _ks_line_element(a, R, T)
    gi = np.linalg.inv(g4)
    det3 = np.linalg.det(g4[..., 1:, 1:])
    sqrtg = np.sqrt(np.maximum(det3, 1e-300))
    alpha = 1.0 / np.sqrt(-gi[..., 0, 0])
    Fup = np.einsum("...am,...bn,...mn->...ab", gi, gi, F)
    D = [alpha * Fup[..., 0, i] for i in (1, 2, 3)]
    B = [F[..., 2, 3] / sqrtg, F[..., 3, 1] / sqrtg, F[..., 1, 2] / sqrtg]
    # on the poles sqrt(gamma) = 0: take the limit from the neighbouring row
    for comp in D + B:
        comp[0, :] = comp[1, :]
        comp[-1, :] = comp[-2, :]
    fields = dict(D=D, B=B, logr0=logr0, dlogr=dlogr, dth=dth, a=a, r_in=r_in, r_out=r_out)
    rng = np.random.default_rng(seed)
    n = n_particles
    lr = rng.uniform(logr0, np.log(r_out), n)
    th = np.arccos(rng.uniform(-1.0, 1.0, n) * 0.98)
    ph = rng.uniform(0.0, 2 * np.pi, n)
    r = np.exp(lr)
    uh = maxwell_juttner(rng, n, theta_mj)
    g4p = _ks_line_element(a, r, th)
    gup = np.linalg.inv(g4p[:, 1:, 1:])
    L = np.linalg.cholesky(gup)                 # gamma^{ij} = L L^T
    u = np.linalg.solve(np.swapaxes(L, 1, 2), uh.T[..., None])[..., 0].T
    state = dict(x=np.ascontiguousarray(np.stack([r, th, ph])), u=np.ascontiguousarray(u),
                 dxp=np.zeros((3, n)), flags=np.zeros(n, dtype=np.uint8))
    params = dict(c=1.0, dt=dt, f_rho=1.0, f_E=1.0, dl=1.0, qm=(qm,), curvature=0,
                  mu_mode=0, grad_mode=0, gca_max_iter=16, gca_fixed_iters=0, gca_tol=1e-7,
                  n_steps=1000, a=a, r_in=r_in, r_out=r_out)
    return fields, state, params
