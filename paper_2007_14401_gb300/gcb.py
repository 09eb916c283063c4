"""ctypes binding of the CUDA C-ABI library ``libgcb.so`` (declared in include/gcb.h).

Argument marshalling only: device memory comes from PyTorch tensors, every
step of the push runs in the library's kernels.  Importing this module loads
the library and raises if it has not been built (no CPU fallback exists).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

F32, F64 = 0, 1
POS_F64, POS_F32PAIR = 0, 1
GRAD_DW, GRAD_GRID = 0, 1
FORCE_NONE, FORCE_BORIS, FORCE_GCA = 0, 1, 2
MU_CONSERVE, UPERP_CONSERVE = 0, 1
FRAME_SIMPLE, FRAME_BT = 0, 1
PHASE_KEEP, PHASE_EVOLVE = 0, 1
MIRROR_OFF, MIRROR_ON = 0, 1
FLAG_S, FLAG_SPREV, FLAG_NONCONV, FLAG_GCAFAIL, FLAG_NONFINITE, FLAG_EXITED = 1, 2, 4, 8, 16, 32
SPECIES_SHIFT = 6
STATUS = {0: "GCB_OK", 1: "GCB_EINVAL", 2: "GCB_ECUDA", 3: "GCB_EUNSUPPORTED", 4: "GCB_ENOMEM"}


class GcbGrid(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("dtype", C.c_int32), ("n", C.c_int64 * 3),
                ("dx", C.c_double * 3), ("has_grad", C.c_int32), ("stride", C.c_int32),
                ("rec", C.c_void_p)]


class GcbParticles(C.Structure):
    _fields_ = [("n", C.c_int64), ("ndim", C.c_int32), ("pos_mode", C.c_int32),
                ("mom_dtype", C.c_int32), ("reserved", C.c_int32), ("x", C.c_void_p * 3),
                ("x_lo", C.c_void_p * 3), ("u", C.c_void_p * 3), ("dxp", C.c_void_p * 3),
                ("flags", C.c_void_p), ("pid", C.c_void_p)]


class GcbParams(C.Structure):
    _fields_ = [("c", C.c_double), ("dt", C.c_double), ("f_rho", C.c_double),
                ("f_E", C.c_double), ("dl", C.c_double), ("qm", C.c_double * 4),
                ("curvature", C.c_int32), ("mu_mode", C.c_int32), ("grad_mode", C.c_int32),
                ("force", C.c_int32), ("gca_max_iter", C.c_int32),
                ("gca_fixed_iters", C.c_int32), ("gca_tol", C.c_double),
                ("sort_every", C.c_int32), ("sort_tile", C.c_int32 * 3),
                ("step_index", C.c_int64), ("fuse_steps", C.c_int32),
                ("drift_frame", C.c_int32), ("gyro_phase", C.c_int32), ("mirror", C.c_int32)]


class GcbStats(C.Structure):
    _fields_ = [("n_boris", C.c_int64), ("n_gca", C.c_int64), ("n_to_gca", C.c_int64),
                ("n_to_boris", C.c_int64), ("n_nonconv", C.c_int64), ("n_gcafail", C.c_int64),
                ("n_nonfinite", C.c_int64), ("sum_iter", C.c_int64), ("max_iter", C.c_int64),
                ("sum_ekin", C.c_double), ("n_exited", C.c_int64)]


class GcbGridKs(C.Structure):
    _fields_ = [("g", GcbGrid), ("logr0", C.c_double), ("dl", C.c_void_p)]


class GcbKsParams(C.Structure):
    _fields_ = [("a", C.c_double), ("r_in", C.c_double), ("r_out", C.c_double),
                ("kick_basis", C.c_int32)]


KS_TETRAD, KS_GLOBAL = 0, 1   # GREOM half kicks in the local frame / the global basis


class GcbCurrent(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("reserved", C.c_int32), ("q", C.c_double * 4),
                ("w", C.c_void_p), ("J", C.c_void_p * 3)]


class GcbDepositStats(C.Structure):
    _fields_ = [("n_skipped", C.c_int64), ("n_pieces", C.c_int64), ("n_atomics", C.c_int64)]


DEPOSIT_MAX_CELLS = 64   # GCB_DEPOSIT_MAX_CELLS


EXPORTS = ["gcb_version", "gcb_status_string", "gcb_last_error", "gcb_grid_stride",
           "gcb_grid_pack", "gcb_pos_split", "gcb_pos_join", "gcb_workspace_bytes",
           "gcb_sort_sr", "gcb_push_sr", "gcb_push_sr_noalloc", "gcb_adjoint_workspace_bytes",
           "gcb_adjoint_sr", "gcb_push_sr_ckpt", "gcb_grid_combine", "gcb_grad_project", "gcb_ks_cell_size",
           "gcb_push_ks", "gcb_push_deposit_sr"]


def load_library(path: str | None = None):
    """Load libgcb.so and declare its signatures (raises if missing)."""
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: call paper_2007_14401_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.POINTER
    lib.gcb_version.restype = C.c_int
    lib.gcb_status_string.argtypes = [C.c_int]
    lib.gcb_status_string.restype = C.c_char_p
    lib.gcb_last_error.restype = C.c_char_p
    lib.gcb_grid_stride.argtypes = [C.c_int32, C.c_int32, C.c_int32]
    lib.gcb_grid_stride.restype = C.c_int32
    lib.gcb_grid_pack.argtypes = [P(GcbGrid), P(C.c_void_p), C.c_void_p]
    lib.gcb_grid_pack.restype = C.c_int
    lib.gcb_pos_split.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.gcb_pos_split.restype = C.c_int
    lib.gcb_pos_join.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.gcb_pos_join.restype = C.c_int
    lib.gcb_workspace_bytes.argtypes = [P(GcbParticles), P(GcbGrid), P(GcbParams)]
    lib.gcb_workspace_bytes.restype = C.c_size_t
    lib.gcb_push_sr.argtypes = [P(GcbParticles), P(GcbGrid), P(GcbParams), C.c_int,
                                C.c_void_p, C.c_void_p, C.c_size_t, P(GcbStats)]
    lib.gcb_push_sr.restype = C.c_int
    lib.gcb_sort_sr.argtypes = [P(GcbParticles), P(GcbGrid), P(GcbParams), C.c_void_p,
                                C.c_void_p, C.c_size_t]
    lib.gcb_sort_sr.restype = C.c_int
    lib.gcb_push_sr_noalloc.argtypes = [P(GcbParticles), P(GcbGrid), P(GcbParams), C.c_int,
                                        C.c_void_p, P(GcbStats)]
    lib.gcb_push_sr_noalloc.restype = C.c_int
    lib.gcb_adjoint_workspace_bytes.argtypes = [P(GcbParticles), P(GcbGrid), P(GcbParams), C.c_int,
                                                C.c_int]
    lib.gcb_adjoint_workspace_bytes.restype = C.c_size_t
    lib.gcb_adjoint_sr.argtypes = [P(GcbParticles), P(GcbGrid), P(GcbParams), C.c_int, C.c_int,
                                   C.c_int, P(C.c_void_p), C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_size_t]
    lib.gcb_adjoint_sr.restype = C.c_int
    lib.gcb_push_sr_ckpt.argtypes = [P(GcbParticles), P(GcbGrid), P(GcbParams), C.c_int, C.c_int,
                                     C.c_void_p, C.c_void_p, C.c_size_t, P(GcbStats)]
    lib.gcb_push_sr_ckpt.restype = C.c_int
    lib.gcb_grid_combine.argtypes = [P(GcbGrid), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                     C.c_void_p]
    lib.gcb_grid_combine.restype = C.c_int
    lib.gcb_grad_project.argtypes = [P(GcbGrid), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                     C.c_void_p]
    lib.gcb_grad_project.restype = C.c_int
    lib.gcb_ks_cell_size.argtypes = [P(GcbGridKs), P(GcbKsParams), C.c_void_p, C.c_void_p]
    lib.gcb_ks_cell_size.restype = C.c_int
    lib.gcb_push_ks.argtypes = [P(GcbParticles), P(GcbGridKs), P(GcbKsParams), P(GcbParams),
                                C.c_int, C.c_void_p, C.c_void_p, C.c_size_t, P(GcbStats)]
    lib.gcb_push_ks.restype = C.c_int
    lib.gcb_push_deposit_sr.argtypes = [P(GcbParticles), P(GcbGrid), P(GcbParams),
                                        P(GcbCurrent), C.c_int, C.c_void_p, C.c_void_p,
                                        C.c_size_t, P(GcbStats), P(GcbDepositStats)]
    lib.gcb_push_deposit_sr.restype = C.c_int
    return lib


_lib = load_library()


def lib():
    return _lib


class GcbError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        msg = _lib.gcb_last_error().decode()
        raise GcbError(f"{what}: {STATUS.get(rc, rc)}: {msg}")


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# --------------------------------------------------------------------------
# field grid
# --------------------------------------------------------------------------
class Grid:
    """A field grid in the library's packed node-record layout (device)."""

    def __init__(self, fields: dict, dtype: str = "f32", device="cuda", stream=None):
        E, B, dB = fields["E"], fields["B"], fields.get("dB")
        shape = np.asarray(E[0]).shape
        self.ndim = len(shape)
        self.n = tuple(reversed(shape)) + (1,) * (3 - len(shape))
        self.dx = tuple(fields["dx"]) + (1.0,) * (3 - self.ndim)
        self.dtype = F32 if dtype == "f32" else F64
        self.has_grad = 1 if dB is not None else 0
        self.stride = _lib.gcb_grid_stride(self.ndim, self.dtype, self.has_grad)
        nn = int(np.prod(shape))
        tdt = torch.float32 if self.dtype == F32 else torch.float64
        self.rec = torch.empty(nn * self.stride, dtype=tdt, device=device)
        comps = list(E) + list(B) + (list(dB) if dB is not None else [])
        dev = [torch.as_tensor(np.ascontiguousarray(c, dtype=np.float64).reshape(-1)).to(device)
               for c in comps]
        self.s = GcbGrid(self.ndim, self.dtype, (C.c_int64 * 3)(*self.n),
                         (C.c_double * 3)(*self.dx), self.has_grad, self.stride,
                         self.rec.data_ptr())
        ptrs = (C.c_void_p * len(dev))(*[t.data_ptr() for t in dev])
        _check(_lib.gcb_grid_pack(C.byref(self.s), ptrs, _stream_ptr(stream)), "gcb_grid_pack")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    @property
    def L(self):
        return tuple(self.n[d] * self.dx[d] for d in range(self.ndim))

    @property
    def shape(self):
        """Node-array shape, (ny, nx) or (nz, ny, nx)."""
        return tuple(reversed(self.n[:self.ndim]))

    def update(self, fields: dict, stream=None):
        """Repack new field values (same grid) into the records in place: the
        time-dependent fields of a PiC step, read by the next push."""
        E, B, dB = fields["E"], fields["B"], fields.get("dB")
        assert np.asarray(E[0]).shape == self.shape and (dB is not None) == bool(self.has_grad)
        comps = list(E) + list(B) + (list(dB) if dB is not None else [])
        dev = [torch.as_tensor(c).reshape(-1).to(self.rec.device, torch.float64)
               for c in comps]
        ptrs = (C.c_void_p * len(dev))(*[t.data_ptr() for t in dev])
        _check(_lib.gcb_grid_pack(C.byref(self.s), ptrs, _stream_ptr(stream)), "gcb_grid_pack")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()


class Current:
    """Current of gcb_push_deposit_sr on a grid's staggered points: J of shape
    (3,) + grid.shape in the particles' momentum type (J_x at (i+1/2, j, k),
    J_y at (i, j+1/2, k), J_z at (i, j, k+1/2), in 2D at the node; each at
    its lower node's index).  q: charge of one macro-particle per species;
    w: optional per-particle weights (tensor of n elements).  Pushes add to J;
    zero() clears it.  Counts summed over the pushes that read them (stats
    on): n_skipped particle-steps left out (paths longer than
    DEPOSIT_MAX_CELLS cells along an axis), n_pieces path pieces deposited,
    n_atomics atomic additions into J."""

    def __init__(self, grid: Grid, q, precision: str = "mixed", w=None, device="cuda"):
        tdt = torch.float64 if precision == "fp64" else torch.float32
        self.dtype = F64 if precision == "fp64" else F32
        self.J = torch.zeros((3,) + grid.shape, dtype=tdt, device=device)
        self.q = tuple(float(v) for v in q) + (0.0,) * (4 - len(q))
        self.w = None if w is None else torch.as_tensor(w).to(device, tdt).contiguous()
        self.n_skipped = self.n_pieces = self.n_atomics = 0

    def zero(self):
        self.J.zero_()
        self.n_skipped = self.n_pieces = self.n_atomics = 0

    def struct(self) -> GcbCurrent:
        s = GcbCurrent()
        s.dtype, s.reserved = self.dtype, 0
        for k in range(4):
            s.q[k] = self.q[k]
        s.w = None if self.w is None else self.w.data_ptr()
        for a in range(3):
            s.J[a] = self.J[a].data_ptr()
        return s


# --------------------------------------------------------------------------
# particle state
# --------------------------------------------------------------------------
class State:
    """Particle state in the library's SoA layout.

    precision "fp64": float64 positions and momenta;  "mixed": float32
    momenta and displacements, positions float64 (pos_mode "f64") or float32
    pairs (pos_mode "pair").  device "cuda" (or "cuda:k") keeps it in device
    memory; "pinned" in pinned host memory, which the kernels read and write
    in place across the host link (include/gcb.h: host-resident particles)."""

    def __init__(self, n, ndim, precision="mixed", pos_mode="pair", device="cuda",
                 with_pid=False):
        self.n, self.ndim, self.precision = int(n), int(ndim), precision
        self.host = device == "pinned"
        self.pos_mode = POS_F32PAIR if (precision == "mixed" and pos_mode == "pair") else POS_F64
        self.mom_dtype = F64 if precision == "fp64" else F32
        mdt = torch.float64 if self.mom_dtype == F64 else torch.float32
        if self.pos_mode == POS_F64:
            self.x = self._alloc((ndim, self.n), torch.float64, device)
            self.x_lo = None
        else:
            self.x = self._alloc((ndim, self.n), torch.float32, device)
            self.x_lo = self._alloc((ndim, self.n), torch.float32, device)
        self.u = self._alloc((3, self.n), mdt, device)
        self.dxp = self._alloc((ndim, self.n), mdt, device)
        self.flags = self._alloc((self.n,), torch.uint8, device)
        self.pid = None
        if with_pid:
            self.pid = self._alloc((self.n,), torch.int64, device)
            self.pid.copy_(torch.arange(self.n, dtype=torch.int64))
        self._make_struct()

    def _alloc(self, shape, dtype, device=None):
        """A buffer the library's kernels can reach for this state: pinned host
        memory for a host-resident state, device memory otherwise."""
        if getattr(self, "host", False):
            return torch.empty(shape, dtype=dtype, device="cpu", pin_memory=True)
        return torch.empty(shape, dtype=dtype, device=device if device else self.u.device)

    def _reachable(self, t: torch.Tensor) -> torch.Tensor:
        """t as a contiguous tensor the kernels can reach (copied if needed)."""
        if self.host:
            if t.is_cuda or not t.is_pinned() or not t.is_contiguous():
                out = self._alloc(tuple(t.shape), t.dtype)
                out.copy_(t)
                return out
            return t
        return t.to(self.u.device).contiguous()

    def _make_struct(self):
        s = GcbParticles()
        s.n, s.ndim, s.pos_mode, s.mom_dtype, s.reserved = (self.n, self.ndim, self.pos_mode,
                                                            self.mom_dtype, 0)
        for d in range(self.ndim):
            s.x[d] = self.x[d].data_ptr()
            s.dxp[d] = self.dxp[d].data_ptr()
            if self.x_lo is not None:
                s.x_lo[d] = self.x_lo[d].data_ptr()
        for k in range(3):
            s.u[k] = self.u[k].data_ptr()
        s.flags = self.flags.data_ptr()
        s.pid = self.pid.data_ptr() if self.pid is not None else None
        self.s = s

    def tensors(self):
        t = [self.x, self.u, self.dxp, self.flags]
        t += [self.x_lo] if self.x_lo is not None else []
        return t + ([self.pid] if self.pid is not None else [])

    @classmethod
    def from_numpy(cls, st: dict, precision="mixed", pos_mode="pair", device="cuda", stream=None,
                   with_pid=False):
        nd, n = st["x"].shape
        self = cls(n, nd, precision, pos_mode, device, with_pid)
        self.load(st, stream)
        return self

    def load(self, st: dict, stream=None):
        """Copy a plain float64 state (oracle layout) into this state."""
        mdt = self.u.dtype
        x64 = self._reachable(torch.as_tensor(np.ascontiguousarray(st["x"], dtype=np.float64)))
        if self.pos_mode == POS_F64:
            self.x.copy_(x64)
        elif self.n:
            for d in range(self.ndim):
                _check(_lib.gcb_pos_split(self.n, C.c_void_p(x64[d].data_ptr()),
                                          C.c_void_p(self.x[d].data_ptr()),
                                          C.c_void_p(self.x_lo[d].data_ptr()), _stream_ptr(stream)),
                       "gcb_pos_split")
        self.u.copy_(torch.as_tensor(np.asarray(st["u"], dtype=np.float64)).to(mdt))
        self.dxp.copy_(torch.as_tensor(np.asarray(st["dxp"], dtype=np.float64)).to(mdt))
        self.flags.copy_(torch.as_tensor(np.asarray(st["flags"], dtype=np.uint8)))
        torch.cuda.synchronize()

    def set_tensors(self, x64: torch.Tensor, u: torch.Tensor, dxp: torch.Tensor,
                    flags: torch.Tensor, stream=None):
        """Fill from tensors: x float64 (ndim, n), u (3, n), dxp (ndim, n)."""
        x64 = self._reachable(x64.to(torch.float64))
        if self.pos_mode == POS_F64:
            self.x.copy_(x64)
        elif self.n:
            for d in range(self.ndim):
                _check(_lib.gcb_pos_split(self.n, C.c_void_p(x64[d].data_ptr()),
                                          C.c_void_p(self.x[d].data_ptr()),
                                          C.c_void_p(self.x_lo[d].data_ptr()), _stream_ptr(stream)),
                       "gcb_pos_split")
        self.u.copy_(u)
        self.dxp.copy_(dxp)
        self.flags.copy_(flags)

    def view(self, lo: int, hi: int) -> "State":
        """Particles lo .. hi-1 as a State sharing this one's memory (for
        streaming particle ranges through the GPU; lo a multiple of 64 keeps
        every array 256-byte aligned)."""
        v = State.__new__(State)
        v.n, v.ndim, v.precision, v.host = int(hi - lo), self.ndim, self.precision, self.host
        v.pos_mode, v.mom_dtype = self.pos_mode, self.mom_dtype
        v.x, v.u, v.dxp, v.flags = (self.x[:, lo:hi], self.u[:, lo:hi], self.dxp[:, lo:hi],
                                    self.flags[lo:hi])
        v.x_lo = self.x_lo[:, lo:hi] if self.x_lo is not None else None
        v.pid = self.pid[lo:hi] if self.pid is not None else None
        v._make_struct()
        return v

    def clone(self) -> "State":
        c = State.__new__(State)
        c.n, c.ndim, c.precision, c.host = self.n, self.ndim, self.precision, self.host

        def cp(t):
            if t is None:
                return None
            if self.host:
                return self._alloc(tuple(t.shape), t.dtype).copy_(t)
            return t.clone()

        c.pos_mode, c.mom_dtype = self.pos_mode, self.mom_dtype
        c.x, c.u, c.dxp, c.flags = cp(self.x), cp(self.u), cp(self.dxp), cp(self.flags)
        c.x_lo, c.pid = cp(self.x_lo), cp(self.pid)
        c._make_struct()
        return c

    def x_f64(self, stream=None) -> torch.Tensor:
        """Positions as a float64 (ndim, n) tensor, on the state's side (pairs joined)."""
        if self.pos_mode == POS_F64:
            return self.x.clone()
        x = self._alloc((self.ndim, self.n), torch.float64, self.x.device)
        for d in range(self.ndim if self.n else 0):
            _check(_lib.gcb_pos_join(self.n, C.c_void_p(self.x[d].data_ptr()),
                                     C.c_void_p(self.x_lo[d].data_ptr()),
                                     C.c_void_p(x[d].data_ptr()), _stream_ptr(stream)),
                   "gcb_pos_join")
        return x

    def to_numpy(self, stream=None) -> dict:
        """The state as plain float64 arrays (positions joined from pairs)."""
        if self.pos_mode == POS_F64:
            x = self.x.double()
        else:
            x = self._alloc((self.ndim, self.n), torch.float64, self.x.device)
            if self.n:
                for d in range(self.ndim):
                    _check(_lib.gcb_pos_join(self.n, C.c_void_p(self.x[d].data_ptr()),
                                             C.c_void_p(self.x_lo[d].data_ptr()),
                                             C.c_void_p(x[d].data_ptr()), _stream_ptr(stream)),
                           "gcb_pos_join")
        torch.cuda.synchronize()
        out = dict(x=x.cpu().numpy(), u=self.u.double().cpu().numpy(),
                   dxp=self.dxp.double().cpu().numpy(), flags=self.flags.cpu().numpy())
        if self.pid is not None:
            out["pid"] = self.pid.cpu().numpy()
        return out


# --------------------------------------------------------------------------
# parameters and the push
# --------------------------------------------------------------------------
def make_params(p: dict, **over) -> GcbParams:
    q = dict(p)
    q.update(over)
    qm = list(q["qm"]) + [0.0] * (4 - len(q["qm"]))
    tile = list(q.get("sort_tile", (0, 0, 0))) + [0, 0, 0]
    return GcbParams(q.get("c", 1.0), q["dt"], q.get("f_rho", 0.4), q.get("f_E", 1.0),
                     q.get("dl", 1.0), (C.c_double * 4)(*qm), int(q.get("curvature", 1)),
                     int(q.get("mu_mode", 0)), int(q.get("grad_mode", 0)), int(q.get("force", 0)),
                     int(q.get("gca_max_iter", 16)), int(q.get("gca_fixed_iters", 0)),
                     float(q.get("gca_tol", 1e-7)), int(q.get("sort_every", 0)),
                     (C.c_int32 * 3)(*tile[:3]), int(q.get("step_index", 0)),
                     int(q.get("fuse_steps", 0)), int(q.get("drift_frame", 0)),
                     int(q.get("gyro_phase", 0)), int(q.get("mirror", 0)))


def _work_device(state):
    """The device of a state's workspace (a host-resident state's: the current GPU)."""
    return "cuda" if getattr(state, "host", False) else state.x.device


class Workspace:
    def __init__(self, state: State, grid: Grid, params: GcbParams, device="cuda"):
        nb = _lib.gcb_workspace_bytes(C.byref(state.s), C.byref(grid.s), C.byref(params))
        self.buf = torch.empty(max(256, (nb + 255) // 256 * 256), dtype=torch.uint8, device=device)
        self.nbytes = self.buf.numel()


def sort(state: State, grid: Grid, params: GcbParams, stream=None,
         workspace: Workspace | None = None):
    """Reorder the particles by cell tile in place (pid follows)."""
    if workspace is None:
        q = GcbParams.from_buffer_copy(params)
        q.sort_every = max(1, q.sort_every)
        workspace = Workspace(state, grid, q, _work_device(state))
    rc = _lib.gcb_sort_sr(C.byref(state.s), C.byref(grid.s), C.byref(params), _stream_ptr(stream),
                          C.c_void_p(workspace.buf.data_ptr()), workspace.nbytes)
    _check(rc, "gcb_sort_sr")


def push(state: State, grid: Grid, params: GcbParams, n_steps: int = 1, stream=None,
         workspace: Workspace | None = None, stats: bool = True,
         current: Current | None = None):
    """Advance ``state`` by n_steps coupled steps in place; returns the stats
    dict (synchronizing the stream) when ``stats`` is true, else None.  With
    ``current`` every step's current is added to current.J
    (gcb_push_deposit_sr; its skip count is read when ``stats``)."""
    ws = workspace or Workspace(state, grid, params, _work_device(state))
    out = GcbStats() if stats else None
    if current is None:
        rc = _lib.gcb_push_sr(C.byref(state.s), C.byref(grid.s), C.byref(params), int(n_steps),
                              _stream_ptr(stream), C.c_void_p(ws.buf.data_ptr()), ws.nbytes,
                              C.byref(out) if stats else None)
        _check(rc, "gcb_push_sr")
    else:
        cs = current.struct()
        dst = GcbDepositStats()
        rc = _lib.gcb_push_deposit_sr(C.byref(state.s), C.byref(grid.s), C.byref(params),
                                      C.byref(cs), int(n_steps), _stream_ptr(stream),
                                      C.c_void_p(ws.buf.data_ptr()), ws.nbytes,
                                      C.byref(out) if stats else None,
                                      C.byref(dst) if stats else None)
        _check(rc, "gcb_push_deposit_sr")
        current.n_skipped += int(dst.n_skipped)
        current.n_pieces += int(dst.n_pieces)
        current.n_atomics += int(dst.n_atomics)
    if stats:
        return {k: getattr(out, k) for k, _ in GcbStats._fields_}
    return None


class StepGraph:
    """n_steps pushes of one state captured in a CUDA graph, replayed with
    one launch of the graph: for small problems, whose steps are short
    enough that issuing them one by one from the host leaves the GPU idle.

    The capture records the calls as they are made now: step p.step_index +
    k for k < n_steps (so the sort schedule of those indices), the state's,
    grid's, workspace's and current's device addresses, and no statistics
    (a call with statistics synchronizes, which a capture cannot).  Each
    replay advances the state by the same n_steps, with the same step
    indices; with sorting, make n_steps a multiple of params.sort_every.
    Push the state once without the graph before capturing (the first call
    of each kernel sizes its grid).  With ``current``, each step adds its
    current to current.J (zero it between replays as a PiC loop would)."""

    def __init__(self, state: State, grid: Grid, params: GcbParams, n_steps: int,
                 workspace: Workspace, current: Current | None = None):
        if n_steps < 1:
            raise ValueError("n_steps must be >= 1")
        self.n_steps = int(n_steps)
        self.graph = torch.cuda.CUDAGraph()
        first = int(params.step_index)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                for k in range(self.n_steps):
                    params.step_index = first + k
                    push(state, grid, params, 1, workspace=workspace, stats=False,
                         current=current)
        params.step_index = first
        torch.cuda.current_stream().wait_stream(side)

    def replay(self):
        """Run the captured steps on the current stream (asynchronous)."""
        self.graph.replay()


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------
LAM_ORDER = ("x0", "x1", "u0", "u1", "u2", "dxp0", "dxp1")


ADJ_METHODS = {"reverse": 0, "tangent": 1}
ADJ_HAVE_CKPT = 0x100


class AdjointWorkspace:
    """Device workspace of the adjoint (checkpoints and segment states) for a
    given state layout, grid, n_steps and checkpoint spacing."""

    def __init__(self, state: State, grid: Grid, n_steps: int, ckpt_every: int = 16,
                 params: GcbParams | None = None):
        nb = _lib.gcb_adjoint_workspace_bytes(C.byref(state.s), C.byref(grid.s),
                                              C.byref(params) if params is not None else None,
                                              int(n_steps), int(ckpt_every))
        if nb == 0:
            raise GcbError("gcb_adjoint_workspace_bytes: invalid arguments")
        self.buf = torch.empty(nb, dtype=torch.uint8, device=state.u.device)
        self.n_steps, self.ckpt_every = int(n_steps), int(ckpt_every)
        self.have_ckpt = False


def push_ckpt(state: State, grid: Grid, params: GcbParams, n_steps: int,
              workspace: AdjointWorkspace, stream=None, stats: bool = False):
    """n_steps pushes of ``state`` in place that also store the adjoint's
    checkpoints in ``workspace`` (for a following adjoint(..., workspace=))."""
    out = GcbStats() if stats else None
    rc = _lib.gcb_push_sr_ckpt(C.byref(state.s), C.byref(grid.s), C.byref(params), int(n_steps),
                               workspace.ckpt_every, _stream_ptr(stream),
                               C.c_void_p(workspace.buf.data_ptr()), workspace.buf.numel(),
                               C.byref(out) if stats else None)
    _check(rc, "gcb_push_sr_ckpt")
    workspace.have_ckpt = True
    if stats:
        return {k: getattr(out, k) for k, _ in GcbStats._fields_}
    return None


def adjoint(state: State, grid: Grid, params: GcbParams, n_steps: int, lam: torch.Tensor,
            ckpt_every: int = 16, stream=None, method: str = "reverse",
            workspace: AdjointWorkspace | None = None) -> torch.Tensor:
    """Reverse sweep of n_steps pushes from the initial ``state`` (left
    unchanged).  ``lam`` (7, n) in the momentum dtype holds dL/d(final x0, x1,
    u0, u1, u2, dxp0, dxp1) and is overwritten with dL/d(initial state).
    Returns dL/d(record values) as a float64 tensor (nodes, 12).  method
    "reverse" (default) or "tangent" (dual-number Jacobian columns, slower).
    A ``workspace`` filled by push_ckpt supplies the checkpoints (and its
    n_steps / ckpt_every must match); otherwise the forward is rerun here."""
    if workspace is None:
        workspace = AdjointWorkspace(state, grid, n_steps, ckpt_every, params)
    elif (workspace.n_steps, workspace.ckpt_every) != (int(n_steps), int(ckpt_every)):
        raise GcbError("workspace was sized for another n_steps / ckpt_every")
    ws, nb = workspace.buf, workspace.buf.numel()
    mcode = ADJ_METHODS[method] | (ADJ_HAVE_CKPT if workspace.have_ckpt else 0)
    nn = grid.n[0] * grid.n[1] * grid.n[2]
    grad = torch.empty((nn, 12), dtype=torch.float64, device=state.u.device)
    if lam.shape != (7, state.n) or lam.dtype != state.u.dtype or not lam.is_contiguous():
        raise GcbError("lam must be a contiguous (7, n) tensor of the momentum dtype")
    ptrs = (C.c_void_p * 7)(*[lam[k].data_ptr() for k in range(7)])
    rc = _lib.gcb_adjoint_sr(C.byref(state.s), C.byref(grid.s), C.byref(params), int(n_steps),
                             int(ckpt_every), mcode, ptrs,
                             C.c_void_p(grad.data_ptr()),
                             _stream_ptr(stream), C.c_void_p(ws.data_ptr()), nb)
    _check(rc, "gcb_adjoint_sr")
    return grad


def grid_combine(grid: Grid, base: torch.Tensor, pat: torch.Tensor, amps: torch.Tensor,
                 stream=None):
    """grid.rec = base + sum_m amps[m] pat[m] (records in grid's layout)."""
    amps = amps.to(device=grid.rec.device, dtype=torch.float64).contiguous()
    rc = _lib.gcb_grid_combine(C.byref(grid.s), C.c_void_p(base.data_ptr()),
                               C.c_void_p(pat.data_ptr()), C.c_void_p(amps.data_ptr()),
                               int(amps.numel()), _stream_ptr(stream))
    _check(rc, "gcb_grid_combine")


def grad_project(grid: Grid, grad: torch.Tensor, pat: torch.Tensor, stream=None) -> torch.Tensor:
    """dL/da_m = <grad, pat[m]> for fields linear in the amplitudes."""
    out = torch.empty(pat.shape[0], dtype=torch.float64, device=grad.device)
    rc = _lib.gcb_grad_project(C.byref(grid.s), C.c_void_p(grad.data_ptr()),
                               C.c_void_p(pat.data_ptr()), int(pat.shape[0]),
                               C.c_void_p(out.data_ptr()), _stream_ptr(stream))
    _check(rc, "gcb_grad_project")
    return out


class ModePush(torch.autograd.Function):
    """Differentiable n-step push: (x0, u0, dxp0, amps) -> (x, u, dxp), the
    field records being base + sum_m amps[m] pat[m].  ``cfg`` is a dict
    with grid, base, pat, params, n_steps, ckpt_every, flags, precision,
    pos_mode, and optionally method and ckpt_in_forward (default True: the
    forward writes the adjoint's checkpoints).  x as float64 (2, n); u (3, n)
    and dxp (2, n) in the momentum dtype."""

    @staticmethod
    def forward(ctx, x0, u0, dxp0, amps, cfg):
        grid = cfg["grid"]
        grid_combine(grid, cfg["base"], cfg["pat"], amps)
        st = State(x0.shape[1], 2, cfg.get("precision", "fp64"), cfg.get("pos_mode", "f64"),
                   device=x0.device)
        st.set_tensors(x0, u0, dxp0, cfg["flags"])
        ctx.cfg = cfg
        if cfg.get("ckpt_in_forward", True):
            # the forward stores the checkpoints; the backward starts from them
            ctx.ws = AdjointWorkspace(st, grid, cfg["n_steps"], cfg.get("ckpt_every", 16),
                                      cfg["params"])
            push_ckpt(st, grid, cfg["params"], cfg["n_steps"], ctx.ws)
            ctx.init = st          # layout only: the initial state is checkpoint 0
        else:
            ctx.ws, ctx.init = None, st.clone()
            # outputs must stay in the inputs' order: no sorting in this push
            # (the adjoint sorts at its checkpoints and restores the order)
            fwd = GcbParams.from_buffer_copy(cfg["params"])
            fwd.sort_every = 0
            push(st, grid, fwd, cfg["n_steps"], stats=False)
        return st.x_f64(), st.u.clone(), st.dxp.clone()

    @staticmethod
    def backward(ctx, gx, gu, gdxp):
        cfg, st = ctx.cfg, ctx.init
        n = st.n
        lam = torch.zeros((7, n), dtype=st.u.dtype, device=st.u.device)
        if gx is not None:
            lam[0:2] = gx.to(lam.dtype)
        if gu is not None:
            lam[2:5] = gu.to(lam.dtype)
        if gdxp is not None:
            lam[5:7] = gdxp.to(lam.dtype)
        grad = adjoint(st, cfg["grid"], cfg["params"], cfg["n_steps"], lam,
                       cfg.get("ckpt_every", 16), method=cfg.get("method", "reverse"),
                       workspace=ctx.ws)
        ga = grad_project(cfg["grid"], grad, cfg["pat"])
        return lam[0:2].to(torch.float64), lam[2:5].clone(), lam[5:7].clone(), ga, None


# --------------------------------------------------------------------------
# covariant (Kerr-Schild) scheme
# --------------------------------------------------------------------------
class KsGrid:
    """Kerr-Schild field records on the (log r, theta) grid plus the cell-size
    table of Eq. (volint), both on the device."""

    def __init__(self, fields: dict, a: float, r_in: float, r_out: float, dtype: str = "f32",
                 device="cuda", stream=None, kick_basis: int = KS_TETRAD):
        nth, nr = np.asarray(fields["D"][0]).shape
        self.dtype = F32 if dtype == "f32" else F64
        self.stride = _lib.gcb_grid_stride(2, self.dtype, 0)
        tdt = torch.float32 if self.dtype == F32 else torch.float64
        self.rec = torch.empty(nr * nth * self.stride, dtype=tdt, device=device)
        comps = list(fields["D"]) + list(fields["B"])
        dev = [torch.as_tensor(np.ascontiguousarray(c, dtype=np.float64).reshape(-1)).to(device)
               for c in comps]
        g = GcbGrid(2, self.dtype, (C.c_int64 * 3)(nr, nth, 1),
                    (C.c_double * 3)(fields["dlogr"], np.pi / (nth - 1), 1.0), 0, self.stride,
                    self.rec.data_ptr())
        ptrs = (C.c_void_p * 6)(*[t.data_ptr() for t in dev])
        _check(_lib.gcb_grid_pack(C.byref(g), ptrs, _stream_ptr(stream)), "gcb_grid_pack")
        self.dl = torch.empty((nth - 1) * (nr - 1), dtype=torch.float64, device=device)
        self.s = GcbGridKs(g, fields["logr0"], self.dl.data_ptr())
        self.kp = GcbKsParams(a, r_in, r_out, kick_basis)
        _check(_lib.gcb_ks_cell_size(C.byref(self.s), C.byref(self.kp),
                                     C.c_void_p(self.dl.data_ptr()), _stream_ptr(stream)),
               "gcb_ks_cell_size")
        torch.cuda.synchronize()
        self._keep = dev


def ks_workspace(device="cuda") -> Workspace:
    """The workspace gcb_push_ks needs (its statistics counters only)."""
    ws = Workspace.__new__(Workspace)
    ws.buf = torch.empty(256, dtype=torch.uint8, device=device)
    ws.nbytes = 256
    return ws


def push_ks(state: State, grid: KsGrid, params: GcbParams, n_steps: int = 1, stream=None,
            workspace: Workspace | None = None, stats: bool = True):
    """n_steps covariant coupled steps of ``state`` (FP64, ndim 3) in place."""
    if workspace is None:
        workspace = ks_workspace(_work_device(state))
    out = GcbStats() if stats else None
    rc = _lib.gcb_push_ks(C.byref(state.s), C.byref(grid.s), C.byref(grid.kp), C.byref(params),
                          int(n_steps), _stream_ptr(stream), C.c_void_p(workspace.buf.data_ptr()),
                          workspace.nbytes, C.byref(out) if stats else None)
    _check(rc, "gcb_push_ks")
    if stats:
        return {k: getattr(out, k) for k, _ in GcbStats._fields_}
    return None
