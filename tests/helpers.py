"""Shared test helpers: oracle wiring for the generated workloads and the
comparison rules of the parity tests."""
import math

import numpy as np

import oracle as O


def oracle_field(fields):
    return O.grid_field(fields["E"], fields["B"], fields["dx"], dB=fields.get("dB"))


def oracle_params(p, **over):
    q = dict(p)
    q.update(over)
    return O.make_params(c=q.get("c", 1.0), dt=q["dt"], f_rho=q.get("f_rho", 0.4),
                         f_E=q.get("f_E", 1.0), dl=q.get("dl", 1.0), qm=tuple(q["qm"]),
                         curvature=q.get("curvature", 1), mu_mode=q.get("mu_mode", 0),
                         grad_mode=q.get("grad_mode", 0), force=q.get("force", 0),
                         max_iter=q.get("gca_max_iter", 16),
                         fixed_iters=q.get("gca_fixed_iters", 0), tol=q.get("gca_tol", 1e-7),
                         frame=q.get("drift_frame", 0), gyro_phase=q.get("gyro_phase", 0),
                         mirror=q.get("mirror", 0))


def copy_state(st):
    return {k: v.copy() for k, v in st.items()}


def switch_margins(ofield, oparams, st):
    """Criterion margin of every particle at its current x and u (oracle)."""
    n = st["flags"].shape[0]
    m = np.empty(n)
    for i in range(n):
        if not (np.all(np.isfinite(st["x"][:, i])) and np.all(np.isfinite(st["u"][:, i]))):
            m[i] = np.inf
            continue
        F = O.eval_field(ofield, oparams, st["x"][:, i])
        qm = oparams.qm[(int(st["flags"][i]) >> 6) & 3]
        G = math.sqrt(1.0 + float(np.dot(st["u"][:, i], st["u"][:, i])) / oparams.c ** 2)
        _, m[i] = O.switch(F[0:3], F[3:6], G, abs(qm), oparams)
    return m


def periodic_diff(a, b, L):
    """a - b for positions, taken modulo the box length per axis."""
    L = np.asarray(L, dtype=float)[:, None]
    d = a - b
    return d - L * np.round(d / L)
