"""FP64 CPU oracle of the coupled guiding-center / Boris pusher (Bacchini et al. 2020).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It wraps the plain C
implementation in ``gcb_oracle.c`` (compiled here with gcc, no CUDA) and shares
no code with the CUDA library.

Arrays use the oracle's own plain layout: positions ``x`` and displacements
``dxp`` of shape (ndim, n), momenta ``u`` of shape (3, n), all float64,
``flags`` uint8 of shape (n,); field components as separate float64 node
arrays of shape (nz, ny, nx) (2D: (ny, nx)).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gcb_oracle.c")
_SRC_KS = os.path.join(_HERE, "gcb_oracle_ks.c")
_HDR = os.path.join(_HERE, "gcb_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

FIELD_GRID, FIELD_UNIFORM, FIELD_HARRIS, FIELD_BOTTLE, FIELD_ROTOR = 0, 1, 2, 3, 4
FRAME_SIMPLE, FRAME_BT = 0, 1
GRAD_DW, GRAD_GRID = 0, 1
FORCE_NONE, FORCE_BORIS, FORCE_GCA = 0, 1, 2
MU_CONSERVE, UPERP_CONSERVE = 0, 1
FLAG_S, FLAG_SPREV, FLAG_NONCONV, FLAG_GCAFAIL, FLAG_NONFINITE, FLAG_EXITED = 1, 2, 4, 8, 16, 32
KS_GRID, KS_VACUUM, KS_MONOPOLE = 0, 1, 2

_SRC_GRAD = os.path.join(_HERE, "gcb_oracle_grad.cpp")
_LIB_GRAD = os.path.join(_BUILD, "liboracle_grad.so")

_lock = threading.Lock()
_lib = None
_lib_grad = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP); returns its path.

    ``GCB_ORACLE_LIB`` names a prebuilt library to load instead; the mutation
    test uses it to run the pins against an oracle with a planted mistake."""
    alt = os.environ.get("GCB_ORACLE_LIB")
    if alt:
        return alt
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_LIB) or max(
        os.path.getmtime(_SRC), os.path.getmtime(_SRC_KS),
        os.path.getmtime(_HDR)) > os.path.getmtime(_LIB)
    if stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, _SRC_KS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def build_grad(force: bool = False) -> str:
    """Compile the dual-number gradient oracle (g++, OpenMP) into its own
    library; returns its path.  ``GCB_ORACLE_GRAD_LIB`` names a prebuilt
    library to load instead (the mutation test's planted mistakes)."""
    alt = os.environ.get("GCB_ORACLE_GRAD_LIB")
    if alt:
        return alt
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_LIB_GRAD) or max(
        os.path.getmtime(_SRC_GRAD), os.path.getmtime(_HDR)) > os.path.getmtime(_LIB_GRAD)
    if stale:
        tmp = _LIB_GRAD + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
               _SRC_GRAD, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_GRAD)
    return _LIB_GRAD


class Field(C.Structure):
    _fields_ = [("kind", C.c_int), ("ndim", C.c_int), ("n", C.c_long * 3),
                ("dx", C.c_double * 3), ("E", C.c_void_p * 3), ("B", C.c_void_p * 3),
                ("dB", C.c_void_p * 9), ("par", C.c_double * 16)]


class Params(C.Structure):
    _fields_ = [("c", C.c_double), ("dt", C.c_double), ("f_rho", C.c_double),
                ("f_E", C.c_double), ("dl", C.c_double), ("qm", C.c_double * 4),
                ("curvature", C.c_int), ("mu_mode", C.c_int), ("grad_mode", C.c_int),
                ("force", C.c_int), ("max_iter", C.c_int), ("fixed_iters", C.c_int),
                ("tol", C.c_double), ("frame", C.c_int), ("gyro_phase", C.c_int),
                ("mirror", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_boris", C.c_long), ("n_gca", C.c_long), ("n_to_gca", C.c_long),
                ("n_to_boris", C.c_long), ("n_nonconv", C.c_long), ("n_gcafail", C.c_long),
                ("n_nonfinite", C.c_long), ("sum_iter", C.c_long), ("max_iter", C.c_long),
                ("sum_ekin", C.c_double), ("n_exited", C.c_long)]


class Detail(C.Structure):
    _fields_ = [("S", C.c_int), ("margin", C.c_double), ("branch", C.c_int),
                ("gcafail", C.c_int), ("nonconv", C.c_int), ("iters", C.c_int),
                ("resid", C.c_double), ("H", C.c_double), ("upar_old", C.c_double),
                ("upar_new", C.c_double), ("mu", C.c_double), ("uperp", C.c_double),
                ("Gamma_full", C.c_double), ("Gamma1", C.c_double), ("k1", C.c_double),
                ("k2", C.c_double), ("k3", C.c_double), ("Rn", C.c_double * 3),
                ("Rnp1", C.c_double * 3), ("bpg", C.c_double * 3), ("vstep", C.c_double * 3)]


class DepositT(C.Structure):
    _fields_ = [("q", C.c_double * 4), ("w", C.c_void_p), ("J", C.c_void_p * 3),
                ("Jabs", C.c_void_p * 3), ("n_skipped", C.c_long)]


class KsField(C.Structure):
    _fields_ = [("kind", C.c_int), ("nr", C.c_int), ("nth", C.c_int), ("logr0", C.c_double),
                ("dlogr", C.c_double), ("dth", C.c_double), ("D", C.c_void_p * 3),
                ("B", C.c_void_p * 3), ("par", C.c_double * 8)]


class KsParams(C.Structure):
    _fields_ = [("a", C.c_double), ("r_in", C.c_double), ("r_out", C.c_double),
                ("kick_basis", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P, D3 = C.POINTER, C.c_double * 3
            lib.orc_eval_field.argtypes = [P(Field), P(Params), D3, C.c_double * 15]
            lib.orc_switch.argtypes = [D3, D3, C.c_double, C.c_double, P(Params),
                                       P(C.c_double)]
            lib.orc_switch.restype = C.c_int
            lib.orc_bt_frame.argtypes = [D3, D3, C.c_double, C.c_double * 9]
            lib.orc_bt_frame.restype = C.c_int
            lib.orc_step_one.argtypes = [P(Field), P(Params), D3, D3, D3,
                                         P(C.c_ubyte), P(Detail)]
            lib.orc_decompose.argtypes = [P(Field), P(Params), C.c_double, D3, D3,
                                          P(C.c_double), P(C.c_double), P(C.c_double), D3]
            lib.orc_decompose.restype = C.c_int
            lib.orc_reconstruct.argtypes = [P(Field), P(Params), C.c_double, D3,
                                            C.c_double, C.c_double, C.c_double, D3, D3]
            lib.orc_reconstruct.restype = C.c_int
            lib.orc_push_sr.argtypes = [C.c_long, C.c_void_p * 3, C.c_void_p * 3,
                                        C.c_void_p * 3, C.c_void_p, P(Field), P(Params),
                                        C.c_int, C.c_int, P(Stats)]
            lib.orc_push_sr.restype = C.c_int
            lib.orc_push_sr_dep.argtypes = [C.c_long, C.c_void_p * 3, C.c_void_p * 3,
                                            C.c_void_p * 3, C.c_void_p, P(Field), P(Params),
                                            C.c_int, C.c_int, P(Stats), P(DepositT)]
            lib.orc_push_sr_dep.restype = C.c_int
            lib.orc_deposit.argtypes = [P(Field), D3, D3, C.c_double, C.c_double, C.c_double,
                                        C.c_void_p * 3, C.c_void_p]
            lib.orc_deposit.restype = C.c_int
            lib.orc_push_resolved.argtypes = [C.c_long, C.c_void_p * 3, C.c_void_p * 3,
                                              C.c_void_p, P(Field), P(Params), C.c_double,
                                              C.c_double, C.c_int]
            lib.orc_push_resolved.restype = C.c_int
            lib.orc_ks_metric.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double * 64]
            lib.orc_ks_gather.argtypes = [P(KsField), C.c_double, C.c_double, D3, D3]
            lib.orc_ks_cell_sizes.argtypes = [P(KsField), C.c_double, C.c_void_p]
            lib.orc_ks_frame.argtypes = [C.c_double, C.c_double, C.c_double, D3, D3,
                                         C.c_double * 6]
            lib.orc_ks_kick.argtypes = [C.c_double, C.c_double, C.c_double, D3, D3, C.c_double,
                                        C.c_double, C.c_int, D3]
            lib.orc_ks_step_one.argtypes = [P(KsField), P(KsParams), P(Params), C.c_void_p,
                                            D3, D3, P(C.c_ubyte), P(Detail)]
            lib.orc_push_ks.argtypes = [C.c_long, C.c_void_p * 3, C.c_void_p * 3, C.c_void_p,
                                        P(KsField), P(KsParams), P(Params), C.c_void_p,
                                        C.c_int, C.c_int, P(Stats)]
            lib.orc_push_ks.restype = C.c_int
            _lib = lib
    return _lib


def make_params(*, c=1.0, dt, f_rho=0.4, f_E=1.0, dl=1.0, qm=(-1.0, 1.0, 0.0, 0.0),
                curvature=1, mu_mode=MU_CONSERVE, grad_mode=GRAD_DW, force=FORCE_NONE,
                max_iter=16, fixed_iters=0, tol=1e-7, frame=0, gyro_phase=0,
                mirror=0) -> Params:
    q = list(qm) + [0.0] * (4 - len(qm))
    return Params(c, dt, f_rho, f_E, dl, (C.c_double * 4)(*q), curvature, mu_mode,
                  grad_mode, force, max_iter, fixed_iters, tol, frame, gyro_phase, mirror)


class OracleField:
    """A field the oracle can evaluate; keeps its numpy arrays alive."""

    def __init__(self, kind, ndim, n=(1, 1, 1), dx=(1.0, 1.0, 1.0), E=None, B=None,
                 dB=None, par=()):
        self._keep = []
        s = Field()
        s.kind, s.ndim = kind, ndim
        n = tuple(n) + (1,) * (3 - len(n))
        dx = tuple(dx) + (1.0,) * (3 - len(dx))
        for k in range(3):
            s.n[k] = int(n[k])
            s.dx[k] = float(dx[k])
        if kind == FIELD_GRID:
            for k in range(3):
                e = np.ascontiguousarray(E[k], dtype=np.float64)
                b = np.ascontiguousarray(B[k], dtype=np.float64)
                assert e.size == n[0] * n[1] * n[2] and b.size == e.size
                self._keep += [e, b]
                s.E[k] = e.ctypes.data
                s.B[k] = b.ctypes.data
            if dB is not None:
                for ij in range(3 * ndim):
                    g = np.ascontiguousarray(dB[ij], dtype=np.float64)
                    self._keep.append(g)
                    s.dB[ij] = g.ctypes.data
        par = list(par) + [0.0] * (16 - len(par))
        for k in range(16):
            s.par[k] = float(par[k])
        self.s = s
        self.ndim = ndim


def grid_field(E, B, dx, dB=None) -> OracleField:
    """Grid field from component arrays E[3], B[3] (each (ny,nx) or (nz,ny,nx))."""
    shape = np.asarray(E[0]).shape
    ndim = len(shape)
    n = tuple(reversed(shape))
    return OracleField(FIELD_GRID, ndim, n, dx, E=E, B=B, dB=dB)


def uniform_field(E, B, ndim=3) -> OracleField:
    return OracleField(FIELD_UNIFORM, ndim, par=list(E) + list(B))


def harris_field(B0, delta, Bg, Ez, y0=0.0) -> OracleField:
    return OracleField(FIELD_HARRIS, 2, par=[B0, delta, Bg, Ez, y0])


def bottle_field(B0, L, E=(0.0, 0.0, 0.0)) -> OracleField:
    return OracleField(FIELD_BOTTLE, 3, par=[B0, L] + list(E))


def rotor_field(B0, k, E0, ndim=3) -> OracleField:
    return OracleField(FIELD_ROTOR, ndim, par=[B0, k, E0])


def bt_frame(E, B, c=1.0):
    """The exact drift frame of (E, B): (v_E, b*, kappa, E', B')."""
    lib = _load()
    out = (C.c_double * 9)()
    ok = lib.orc_bt_frame((C.c_double * 3)(*E), (C.c_double * 3)(*B), c, out)
    if not ok:
        raise ValueError("B = 0")
    v = np.array(out[:])
    return v[0:3], v[3:6], v[6], v[7], v[8]


def eval_field(field: OracleField, params: Params, x) -> np.ndarray:
    lib = _load()
    out = (C.c_double * 15)()
    xx = (C.c_double * 3)(*(list(x) + [0.0] * (3 - len(x))))
    lib.orc_eval_field(C.byref(field.s), C.byref(params), xx, out)
    return np.array(out[:])


def switch(E, B, Gam, Q, params: Params):
    lib = _load()
    m = C.c_double()
    S = lib.orc_switch((C.c_double * 3)(*E), (C.c_double * 3)(*B), Gam, Q,
                       C.byref(params), C.byref(m))
    return S, m.value


def step_one(field: OracleField, params: Params, x, u, dxp, flags=0):
    """One coupled step of one particle; returns (x, u, dxp, flags, detail)."""
    lib = _load()
    xx = (C.c_double * 3)(*(list(x) + [0.0] * (3 - len(x))))
    uu = (C.c_double * 3)(*u)
    dd = (C.c_double * 3)(*(list(dxp) + [0.0] * (3 - len(dxp))))
    fl = C.c_ubyte(flags)
    det = Detail()
    lib.orc_step_one(C.byref(field.s), C.byref(params), xx, uu, dd, C.byref(fl),
                     C.byref(det))
    nd = field.ndim
    return np.array(xx[:nd]), np.array(uu[:]), np.array(dd[:nd]), fl.value, det


def decompose(field, params, qm, R, u):
    lib = _load()
    up, mu, uperp = C.c_double(), C.c_double(), C.c_double()
    bpg = (C.c_double * 3)()
    ok = lib.orc_decompose(C.byref(field.s), C.byref(params), qm,
                           (C.c_double * 3)(*(list(R) + [0.0] * (3 - len(R)))),
                           (C.c_double * 3)(*u), C.byref(up), C.byref(mu),
                           C.byref(uperp), bpg)
    return ok, up.value, mu.value, uperp.value, np.array(bpg[:])


def reconstruct(field, params, qm, R, upar, mu, uperp, bpg):
    lib = _load()
    u = (C.c_double * 3)()
    ok = lib.orc_reconstruct(C.byref(field.s), C.byref(params), qm,
                             (C.c_double * 3)(*(list(R) + [0.0] * (3 - len(R)))),
                             upar, mu, uperp, (C.c_double * 3)(*bpg), u)
    return ok, np.array(u[:])


def _ptrs(arrs, k):
    p = (C.c_void_p * 3)()
    for i in range(k):
        assert arrs[i].dtype == np.float64 and arrs[i].flags.c_contiguous
        p[i] = arrs[i].ctypes.data
    return p


DEP_MAX_CELLS = 64


class Current:
    """Current grid of the oracle's deposition: J[a] float64 node arrays of
    the field's shape, J_x at (i+1/2, j, k), J_y at (i, j+1/2, k), J_z at
    (i, j, k+1/2) (2D: at the node), each stored at its lower node's index;
    Jabs[a] the sum of the absolute contributions (the scale of its rounding).
    q: charge of one macro-particle per species; w: per-particle weights or
    None (1)."""

    def __init__(self, shape, q, w=None):
        self.J = [np.zeros(shape) for _ in range(3)]
        self.Jabs = [np.zeros(shape) for _ in range(3)]
        self.q = tuple(q) + (0.0,) * (4 - len(q))
        self.w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        self.n_skipped = 0

    def struct(self):
        d = DepositT()
        for k in range(4):
            d.q[k] = self.q[k]
        d.w = None if self.w is None else self.w.ctypes.data
        for a in range(3):
            d.J[a] = self.J[a].ctypes.data
            d.Jabs[a] = self.Jabs[a].ctypes.data
        return d


def deposit(field: OracleField, x0, disp, vz, Qw, dt, cur: Current) -> bool:
    """Add one particle-step's current (path x0 -> x0 + disp, out-of-plane
    velocity vz in 2D) to ``cur``; False when the path is too long."""
    lib = _load()
    nd = field.ndim
    J = (C.c_void_p * 3)(*[cur.J[a].ctypes.data for a in range(3)])
    Ja = (C.c_void_p * 3)(*[cur.Jabs[a].ctypes.data for a in range(3)])
    rc = lib.orc_deposit(C.byref(field.s), (C.c_double * 3)(*(list(x0[:nd]) + [0.0] * (3 - nd))),
                         (C.c_double * 3)(*(list(disp[:nd]) + [0.0] * (3 - nd))), vz, Qw, dt, J,
                         C.cast(Ja, C.c_void_p))
    return rc == 0


def push_sr(state: dict, field: OracleField, params: Params, n_steps: int,
            nthreads: int = 0, current: Current | None = None) -> dict:
    """Advance ``state`` (dict x, u, dxp, flags; modified in place) by n_steps;
    with ``current``, every step's current is added to it."""
    lib = _load()
    x, u, dxp, flags = state["x"], state["u"], state["dxp"], state["flags"]
    nd = field.ndim
    n = flags.shape[0]
    assert x.shape == (nd, n) and u.shape == (3, n) and dxp.shape == (nd, n)
    assert flags.dtype == np.uint8 and flags.flags.c_contiguous
    xs = [x[k] for k in range(nd)]
    us = [u[k] for k in range(3)]
    ds = [dxp[k] for k in range(nd)]
    st = Stats()
    if current is None:
        rc = lib.orc_push_sr(n, _ptrs(xs, nd), _ptrs(us, 3), _ptrs(ds, nd),
                             flags.ctypes.data, C.byref(field.s), C.byref(params),
                             n_steps, nthreads, C.byref(st))
    else:
        assert current.w is None or current.w.shape == (n,)
        d = current.struct()
        rc = lib.orc_push_sr_dep(n, _ptrs(xs, nd), _ptrs(us, 3), _ptrs(ds, nd),
                                 flags.ctypes.data, C.byref(field.s), C.byref(params),
                                 n_steps, nthreads, C.byref(st), C.byref(d))
        current.n_skipped += d.n_skipped
    if rc != 0:
        raise RuntimeError(f"orc_push_sr failed ({rc})")
    return {k: getattr(st, k) for k, _ in Stats._fields_}


def push_resolved(state: dict, field: OracleField, params: Params, t_end: float,
                  dt_max: float, nthreads: int = 0) -> None:
    """Gyro-resolved Boris reference (adaptive dt = 2 pi / (60 Omega_C))."""
    lib = _load()
    x, u, flags = state["x"], state["u"], state["flags"]
    nd = field.ndim
    n = flags.shape[0]
    rc = lib.orc_push_resolved(n, _ptrs([x[k] for k in range(nd)], nd),
                               _ptrs([u[k] for k in range(3)], 3), flags.ctypes.data,
                               C.byref(field.s), C.byref(params), t_end, dt_max,
                               nthreads)
    if rc != 0:
        raise RuntimeError("orc_push_resolved failed")


# --------------------------------------------------------------------------
# Kerr-Schild (covariant) scheme
# --------------------------------------------------------------------------
class OracleKsField:
    """A Kerr-Schild field for the oracle (keeps its arrays alive)."""

    def __init__(self, kind, nr=2, nth=2, logr0=0.0, dlogr=1.0, D=None, B=None, par=()):
        self._keep = []
        s = KsField()
        s.kind, s.nr, s.nth = kind, nr, nth
        s.logr0, s.dlogr = logr0, dlogr
        s.dth = np.pi / (nth - 1)
        if kind == KS_GRID:
            for k in range(3):
                d = np.ascontiguousarray(D[k], dtype=np.float64).reshape(-1)
                b = np.ascontiguousarray(B[k], dtype=np.float64).reshape(-1)
                assert d.size == nr * nth and b.size == d.size
                self._keep += [d, b]
                s.D[k] = d.ctypes.data
                s.B[k] = b.ctypes.data
        par = list(par) + [0.0] * (8 - len(par))
        for k in range(8):
            s.par[k] = float(par[k])
        self.s = s
        self.nr, self.nth = nr, nth


def ks_grid_field(fields) -> OracleKsField:
    """From a dict with D, B (lists of (nth, nr) arrays), logr0, dlogr."""
    nth, nr = np.asarray(fields["D"][0]).shape
    return OracleKsField(KS_GRID, nr, nth, fields["logr0"], fields["dlogr"], D=fields["D"],
                         B=fields["B"])


KICK_TETRAD, KICK_GLOBAL = 0, 1


def ks_params(a, r_in, r_out, kick_basis=KICK_TETRAD) -> KsParams:
    return KsParams(a, r_in, r_out, kick_basis)


def ks_metric(a, r, th) -> dict:
    lib = _load()
    out = (C.c_double * 64)()
    lib.orc_ks_metric(a, r, th, out)
    v = np.array(out[:])
    return dict(alpha=v[0], beta=v[1:4], gdn=v[4:13].reshape(3, 3), gup=v[13:22].reshape(3, 3),
                sqrtg=v[22], dalpha=v[23:26], dbeta=v[26:35].reshape(3, 3),
                dgup=v[35:62].reshape(3, 3, 3))


def ks_gather(field: OracleKsField, r, th):
    lib = _load()
    D, B = (C.c_double * 3)(), (C.c_double * 3)()
    lib.orc_ks_gather(C.byref(field.s), r, th, D, B)
    return np.array(D[:]), np.array(B[:])


def ks_cell_sizes(field: OracleKsField, a) -> np.ndarray:
    lib = _load()
    out = np.empty((field.nth - 1, field.nr - 1))
    lib.orc_ks_cell_sizes(C.byref(field.s), a, out.ctypes.data)
    return out


def ks_kick(a, r, th, D, B, qm, dtau, u, basis=KICK_TETRAD) -> np.ndarray:
    """Boris kick (Sec. 2.3) of covariant u by contravariant D, B at (r, theta)
    over proper time dtau, in the local frame or the global coordinate basis."""
    lib = _load()
    uu = (C.c_double * 3)(*u)
    lib.orc_ks_kick(a, r, th, (C.c_double * 3)(*D), (C.c_double * 3)(*B), qm, dtau, int(basis), uu)
    return np.array(uu[:])


def ks_frame(a, r, th, u, F):
    lib = _load()
    out = (C.c_double * 6)()
    lib.orc_ks_frame(a, r, th, (C.c_double * 3)(*u), (C.c_double * 3)(*F), out)
    return np.array(out[:3]), np.array(out[3:])


def ks_step_one(field, kp, params, x, u, flags=0, dl=None):
    lib = _load()
    xx, uu = (C.c_double * 3)(*x), (C.c_double * 3)(*u)
    fl = C.c_ubyte(flags)
    det = Detail()
    dptr = None if dl is None else np.ascontiguousarray(dl, dtype=np.float64)
    lib.orc_ks_step_one(C.byref(field.s), C.byref(kp), C.byref(params),
                        None if dptr is None else dptr.ctypes.data, xx, uu, C.byref(fl),
                        C.byref(det))
    return np.array(xx[:]), np.array(uu[:]), fl.value, det


def push_ks(state: dict, field, kp, params, n_steps, dl=None, nthreads=0) -> dict:
    """Advance state (x (3,n) r,theta,phi; u (3,n) covariant; flags) in place."""
    lib = _load()
    x, u, flags = state["x"], state["u"], state["flags"]
    n = flags.shape[0]
    dptr = None if dl is None else np.ascontiguousarray(dl, dtype=np.float64)
    st = Stats()
    rc = lib.orc_push_ks(n, _ptrs([x[k] for k in range(3)], 3), _ptrs([u[k] for k in range(3)], 3),
                         flags.ctypes.data, C.byref(field.s), C.byref(kp), C.byref(params),
                         None if dptr is None else dptr.ctypes.data, n_steps, nthreads,
                         C.byref(st))
    if rc != 0:
        raise RuntimeError("orc_push_ks failed")
    return {k: getattr(st, k) for k, _ in Stats._fields_}


# --------------------------------------------------------------------------
# dual-number gradient of the flat-space push (gcb_oracle_grad.cpp)
# --------------------------------------------------------------------------
def _load_grad():
    global _lib_grad
    with _lock:
        if _lib_grad is None:
            lib = C.CDLL(build_grad())
            lib.orcg_push_jac.argtypes = [C.c_long, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_long, C.c_long, C.c_double,
                                          C.c_double, C.c_void_p, C.c_void_p, C.c_int,
                                          C.c_void_p, C.POINTER(Params), C.c_int, C.c_int,
                                          C.c_void_p]
            lib.orcg_push_jac.restype = C.c_int
            _lib_grad = lib
    return _lib_grad


REC_ORDER = ("E0", "E1", "E2", "B0", "B1", "B2", "dxB0", "dxB1", "dxB2", "dyB0", "dyB1", "dyB2")


def mode_records(fields) -> np.ndarray:
    """(ny*nx, 12) float64 node records of a 2D field dict with gradient
    grids, in REC_ORDER."""
    comps = list(fields["E"]) + list(fields["B"]) + list(fields["dB"])[:6]
    return np.ascontiguousarray(np.stack([np.asarray(c, dtype=np.float64).reshape(-1)
                                          for c in comps], axis=1))


def push_jac(state: dict, base: dict, patterns: list, amps, params: Params, n_steps: int,
             nthreads: int = 0) -> np.ndarray:
    """n_steps of the 2D push (grad mode GRID) in the field base + sum_m
    amps[m] patterns[m], with the derivatives of every particle's final state
    carried along by dual numbers.  ``state`` (x, u, dxp, flags) is advanced
    in place (the oracle's values); returns the Jacobian (n, 7, M + 3):
    d(final x0, x1, u0, u1, u2, dxp0, dxp1) / d(a_0 .. a_{M-1}, u0_x, u0_y,
    u0_z) of each particle."""
    lib = _load_grad()
    amps = np.ascontiguousarray(amps, dtype=np.float64)
    M = amps.size
    if M > 64:
        raise ValueError("at most 64 mode amplitudes")
    rec = mode_records(base)
    if M:
        pat = np.ascontiguousarray(np.stack([mode_records(q) for q in patterns], axis=2))
    else:
        pat = np.zeros((rec.shape[0], 12, 1))
    ny, nx = np.asarray(base["B"][0]).shape
    x, u, dxp, flags = state["x"], state["u"], state["dxp"], state["flags"]
    n = flags.shape[0]
    for a in (x, u, dxp):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    assert x.shape == (2, n) and u.shape == (3, n) and dxp.shape == (2, n)
    jac = np.zeros((n, 7, M + 3))
    rc = lib.orcg_push_jac(n, x.ctypes.data, u.ctypes.data, dxp.ctypes.data, flags.ctypes.data,
                           nx, ny, float(base["dx"][0]), float(base["dx"][1]),
                           rec.ctypes.data, pat.ctypes.data, M, amps.ctypes.data,
                           C.byref(params), int(n_steps), int(nthreads), jac.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"orcg_push_jac failed ({rc})")
    return jac
